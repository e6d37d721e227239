"""Uniform quantization of the coefficient classes (test infrastructure only).

The paper (Section V-B, lossy compression) runs MGARD's quantization and
de-quantization on the GPU right after the decomposition, between the data
refactoring and the entropy coder, but does not state the quantizer.  This
module is the reading the library implements, written from its definition:

  class of a node: the coefficient class it holds in the in-place layout of
    a decomposition with L levels (Fig. 3): class 0 = the coarsest nodes
    N_0, class l = N_l minus N_{l-1}, i.e. the smallest l whose node set
    (indices multiple of 2^(L-l) in every dimension) contains the node;
  code:  q = sign(c) * floor(|c| * (1 / bin_k) + 1/2) for a node of class k
    (uniform quantizer, rounding half away from zero), evaluated in the
    precision of the field (float32 arithmetic for FP32 fields), so that a
    tie is decided the same way on both sides; codes saturate at
    +-(2^31 - 1);
  de-quantized value: q * bin_k, in the precision of the field.

Plain numpy; float32 inputs stay float32 through the quantizer.
"""
from __future__ import annotations

import numpy as np

CODE_MAX = 2 ** 31 - 1


def node_classes(shape, L: int) -> np.ndarray:
    """int32 array of the class of every node (definition above)."""
    out = np.full(shape, -1, dtype=np.int32)
    for l in range(0, L + 1):  # coarse to fine: a node keeps the first level holding it
        s = 1 << (L - l)
        on = np.ones(shape, dtype=bool)
        for k, n in enumerate(shape):
            sh = [1] * len(shape)
            sh[k] = n
            on &= (np.arange(n) % s == 0).reshape(sh)
        out[(out < 0) & on] = l
    return out


def _bins(bins, L, dt):
    b = np.asarray(bins, dtype=np.float64)
    if b.shape != (L + 1,) or not np.all(b > 0) or not np.all(np.isfinite(b)):
        raise ValueError(f"bins must be L + 1 = {L + 1} positive finite values")
    return b.astype(dt)


def quantize(c: np.ndarray, bins, L: int) -> np.ndarray:
    """int32 codes of the decomposed field c (float32 or float64)."""
    dt = c.dtype
    one, half = dt.type(1), dt.type(0.5)
    b = _bins(bins, L, dt)
    inv = (one / b).astype(dt)            # 1 / bin_k rounded to the field precision
    k = node_classes(c.shape, L)
    a = np.abs(c)
    m = (a * inv[k]).astype(dt)           # one rounding, as the product in the field precision
    r = np.floor((m + half).astype(dt))   # one rounding for the addition
    r = np.minimum(r, np.float64(CODE_MAX))
    q = np.where(c < 0, -r, r).astype(np.float64)
    return q.astype(np.int32)


def dequantize(q: np.ndarray, bins, L: int, dtype) -> np.ndarray:
    """The field precision's q * bin_k for every node."""
    dt = np.dtype(dtype)
    b = _bins(bins, L, dt)
    k = node_classes(q.shape, L)
    return (q.astype(dt) * b[k]).astype(dt)
