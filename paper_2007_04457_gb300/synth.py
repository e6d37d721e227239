"""Seeded synthetic inputs (smooth sinusoid sum plus noise).

These fields stand in for the Gray-Scott reaction-diffusion snapshots the
paper measures on (Section IV-A); the paper notes that the cost of the method
does not depend on the values, only on the grid size.  This module holds no
arithmetic of the decomposition itself: it only produces inputs, and both the
CUDA path and the CPU oracle consume what it returns.

Recipe (numpy PCG64 ``default_rng(seed)``, drawn in this order):
  for each of ``n_modes`` modes: ``freq = rng.integers(1, 9, size=d)``,
  ``amp = rng.uniform(0, 1)``, ``phase = rng.uniform(0, 2*pi)``;
  then ``noise = rng.normal(0, noise_sigma, shape)`` in C order.
  u = sum_m amp_m * sin(2*pi * (freq_m . x) + phase_m) + noise,
  x_k = i_k / (n_k - 1) on [0, 1].  An optional Gaussian blob
  exp(-|x - 0.5|^2 / (2 sigma^2)) with sigma = 0.05 is added on top.
FP32 inputs are the FP64 field rounded to nearest.
"""
from __future__ import annotations

import numpy as np


def uniform_coords(shape):
    """Per-dimension node coordinates i / (n - 1)."""
    return [np.arange(n, dtype=np.float64) / (n - 1) for n in shape]


def draw_modes(d: int, n_modes: int, rng: np.random.Generator):
    modes = []
    for _ in range(n_modes):
        freq = rng.integers(1, 9, size=d)
        amp = rng.uniform(0.0, 1.0)
        phase = rng.uniform(0.0, 2.0 * np.pi)
        modes.append((freq, amp, phase))
    return modes


def _phase_grid(shape, freq):
    """2*pi*(freq . x) as a broadcastable sum of per-axis terms."""
    terms = []
    for k, (n, f) in enumerate(zip(shape, freq)):
        x = np.arange(n, dtype=np.float64) / (n - 1)
        s = [1] * len(shape)
        s[k] = n
        terms.append((2.0 * np.pi * f * x).reshape(s))
    return terms


def sinusoid_field(shape, n_modes: int, seed: int, noise_sigma: float = 1e-3,
                   blob: bool = False, dtype=np.float64) -> np.ndarray:
    """Host field of the recipe above, returned in ``dtype``."""
    shape = tuple(int(n) for n in shape)
    rng = np.random.default_rng(seed)
    modes = draw_modes(len(shape), n_modes, rng)
    u = np.zeros(shape, dtype=np.float64)
    for freq, amp, phase in modes:
        terms = _phase_grid(shape, freq)
        arg = terms[0] + phase
        for t in terms[1:]:
            arg = arg + t
        u += amp * np.sin(arg)
    if noise_sigma > 0:
        u += rng.normal(0.0, noise_sigma, shape)
    if blob:
        r2 = np.zeros(shape, dtype=np.float64)
        for k, n in enumerate(shape):
            s = [1] * len(shape)
            s[k] = n
            r2 = r2 + ((np.arange(n) / (n - 1) - 0.5) ** 2).reshape(s)
        u += np.exp(-r2 / (2.0 * 0.05 ** 2))
    return u.astype(dtype)


def sinusoid_field_torch(shape, n_modes: int, seed: int, device, dtype,
                         noise_sigma: float = 1e-3, blob: bool = False):
    """Same modes as ``sinusoid_field`` evaluated on the device with torch.

    The noise comes from a torch generator seeded with ``seed`` (so it is not
    bit-identical to the host field); used where only the workload's shape
    and value distribution matter, e.g. the throughput benchmark.
    """
    import torch

    shape = tuple(int(n) for n in shape)
    rng = np.random.default_rng(seed)
    modes = draw_modes(len(shape), n_modes, rng)
    u = torch.zeros(shape, dtype=torch.float64 if dtype == torch.float64 else torch.float32,
                    device=device)
    axes = []
    for k, n in enumerate(shape):
        s = [1] * len(shape)
        s[k] = n
        axes.append((torch.arange(n, device=device, dtype=torch.float64) / (n - 1), s))
    for freq, amp, phase in modes:
        arg = None
        for (x, s), f in zip(axes, freq):
            t = (2.0 * np.pi * float(f) * x).reshape(s)
            arg = t if arg is None else arg + t
        u += (amp * torch.sin(arg + phase)).to(u.dtype)
    if noise_sigma > 0:
        g = torch.Generator(device=device)
        g.manual_seed(int(seed))
        u += noise_sigma * torch.randn(shape, generator=g, device=device, dtype=u.dtype)
    if blob:
        r2 = None
        for x, s in axes:
            t = ((x - 0.5) ** 2).reshape(s)
            r2 = t if r2 is None else r2 + t
        u += torch.exp(-r2 / (2.0 * 0.05 ** 2)).to(u.dtype)
    return u.to(dtype)


def batch_shapes(seed: int = 4, n3d: int = 240, n2d: int = 16):
    """Shapes of the uneven batch: n3d cubes with sides drawn uniformly from
    {17, 33, 65, 129, 257}, then n2d fields of 1025 x 1025."""
    rng = np.random.default_rng(seed)
    sides = np.array([17, 33, 65, 129, 257])
    shapes = [(int(s),) * 3 for s in sides[rng.integers(0, len(sides), size=n3d)]]
    shapes += [(1025, 1025)] * n2d
    return shapes


def keep_mask(shape, seed: int = 5, keep: float = 0.1):
    """Mask that keeps a random fraction ``keep`` of the finest-level
    coefficients (nodes with any odd index) and every other node."""
    shape = tuple(int(n) for n in shape)
    rng = np.random.default_rng(seed)
    r = rng.random(shape)
    odd = np.zeros(shape, dtype=bool)
    for k, n in enumerate(shape):
        s = [1] * len(shape)
        s[k] = n
        odd = odd | (np.arange(n) % 2 == 1).reshape(s)
    return np.where(odd, r < keep, True)
