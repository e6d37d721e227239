"""ctypes front end of the FP64 C oracle (``mgard_oracle.c``).

TEST INFRASTRUCTURE ONLY: the correctness reference for the CUDA library.
Arrays are numpy float64, row-major, slowest dimension first.  Every function
returns a new array and leaves its input untouched.

Section II-A, Eq. 1-2 of the paper define what is computed; the C file states
the readings of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mgard_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liboracle.so`` (no -ffast-math)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        for name in ("orc_decompose", "orc_recompose", "orc_decompose_adjoint",
                     "orc_recompose_adjoint"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_int, lp, ctypes.POINTER(dp), ctypes.c_int, dp]
            f.restype = ctypes.c_int
        for name in ("orc_decompose_per_dim", "orc_recompose_per_dim",
                     "orc_decompose_adjoint_per_dim", "orc_recompose_adjoint_per_dim"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_int, lp, ctypes.POINTER(dp), ctypes.POINTER(ctypes.c_int), dp]
            f.restype = ctypes.c_int
        for name in ("orc_line_mass", "orc_line_prolong", "orc_line_restrict"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_long, dp, dp, dp]
            f.restype = None
        lib.orc_line_mass_solve.argtypes = [ctypes.c_long, dp, dp, dp]
        lib.orc_line_mass_solve.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def uniform_coords(n: int) -> np.ndarray:
    """x_i = i / (n - 1) on [0, 1]."""
    return np.arange(n, dtype=np.float64) / (n - 1)


def max_levels(shape) -> int:
    """Largest L with (n_k - 1) divisible by 2^L for every dimension."""
    L = 0
    while all((n - 1) % (1 << (L + 1)) == 0 and (n - 1) >= (1 << (L + 1)) for n in shape):
        L += 1
    return L


def dim_levels(shape) -> tuple:
    """Per dimension, the largest L_k with (n_k - 1) divisible by 2^L_k."""
    out = []
    for n in shape:
        L = 0
        while (n - 1) % (1 << (L + 1)) == 0 and (n - 1) >= (1 << (L + 1)):
            L += 1
        out.append(L)
    return tuple(out)


def _run(fn_name: str, u: np.ndarray, nlevels, coords) -> np.ndarray:
    lib = _load()
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    d = u.ndim
    if not 1 <= d <= 3:
        raise ValueError("oracle supports 1 to 3 dimensions")
    shape = u.shape
    per_dim = fn_name.endswith("_per_dim")
    if per_dim:
        Lk = dim_levels(shape) if nlevels is None else tuple(int(v) for v in nlevels)
        if len(Lk) != d:
            raise ValueError("one level count per dimension")
        L = (ctypes.c_int * d)(*Lk)
    else:
        L = max_levels(shape) if nlevels is None or nlevels < 0 else int(nlevels)
    if coords is None:
        coords = [uniform_coords(n) for n in shape]
    xs = [np.ascontiguousarray(np.asarray(c, dtype=np.float64)) for c in coords]
    if len(xs) != d or any(x.shape != (n,) for x, n in zip(xs, shape)):
        raise ValueError("one coordinate array per dimension, of matching length")
    n_arr = (ctypes.c_long * d)(*shape)
    x_arr = (ctypes.POINTER(ctypes.c_double) * d)(*[_dp(x) for x in xs])
    rc = getattr(lib, fn_name)(d, n_arr, x_arr, L, _dp(u))
    if rc != 0:
        raise ValueError(f"{fn_name} failed with code {rc} (shape {shape}, "
                         f"L={list(L) if per_dim else L})")
    return u


def decompose(u, nlevels=None, coords=None):
    """Multilevel decomposition (Eq. 1), levels L..1, in-place nodal layout."""
    return _run("orc_decompose", u, nlevels, coords)


def recompose(u, nlevels=None, coords=None):
    """Exact inverse of ``decompose``, levels 1..L."""
    return _run("orc_recompose", u, nlevels, coords)


def recompose_classes(u, nclasses, nlevels=None, coords=None):
    """Recomposition from the first ``nclasses`` coefficient classes
    (Section I, Fig. 1: an approximation is rebuilt from a chosen number of
    classes; Section II-A, overall process: the omitted coefficients are left
    out of the recomposition).  Class 0 is the coarsest nodal values on N_0,
    class l the level-l coefficients on N_l \\ N_{l-1}.  Leaving a class out
    means its coefficients are zero: every node outside N_{nclasses-1} is set
    to zero and the full recomposition runs.  1 <= nclasses <= L + 1."""
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    L = max_levels(u.shape) if nlevels is None or nlevels < 0 else int(nlevels)
    if not 1 <= int(nclasses) <= L + 1:
        raise ValueError(f"nclasses must be in 1..{L + 1}")
    stride = 1 << (L - (int(nclasses) - 1))
    kept = np.zeros(u.shape, dtype=bool)
    kept[np.ix_(*[np.arange(0, n, stride) for n in u.shape])] = True
    u[~kept] = 0.0
    return recompose(u, L, coords)


def decompose_per_dim(u, levels=None, coords=None):
    """Decomposition with a level count per dimension (default: each
    dimension's own maximum, ``dim_levels``): dimension k coarsens in the
    first levels[k] steps from the finest level and then keeps its nodes, so
    short sides stop early (a generalisation of the equal sides of Section
    IV; Eq. 1-2 unchanged on the nested tensor-product spaces)."""
    return _run("orc_decompose_per_dim", u, levels, coords)


def recompose_per_dim(u, levels=None, coords=None):
    """Exact inverse of ``decompose_per_dim``."""
    return _run("orc_recompose_per_dim", u, levels, coords)


def decompose_adjoint_per_dim(u, levels=None, coords=None):
    """Transpose of ``decompose_per_dim``."""
    return _run("orc_decompose_adjoint_per_dim", u, levels, coords)


def recompose_adjoint_per_dim(u, levels=None, coords=None):
    """Transpose of ``recompose_per_dim``."""
    return _run("orc_recompose_adjoint_per_dim", u, levels, coords)


def decompose_adjoint(u, nlevels=None, coords=None):
    """Transpose of the linear map ``decompose``."""
    return _run("orc_decompose_adjoint", u, nlevels, coords)


def recompose_adjoint(u, nlevels=None, coords=None):
    """Transpose of the linear map ``recompose``."""
    return _run("orc_recompose_adjoint", u, nlevels, coords)


def line_mass(x, v):
    """M v for the 6x-scaled P1 mass matrix on nodes x."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.empty_like(v)
    lib.orc_line_mass(len(v), _dp(x), _dp(v), _dp(out))
    return out


def line_prolong(xf, vc):
    """P vc: coarse nodes (even fine indices) to all fine nodes xf."""
    lib = _load()
    xf = np.ascontiguousarray(xf, dtype=np.float64)
    vc = np.ascontiguousarray(vc, dtype=np.float64)
    out = np.empty(len(xf), dtype=np.float64)
    lib.orc_line_prolong(len(xf), _dp(xf), _dp(vc), _dp(out))
    return out


def line_restrict(xf, vf):
    """P^T vf: fine nodes xf to the coarse nodes."""
    lib = _load()
    xf = np.ascontiguousarray(xf, dtype=np.float64)
    vf = np.ascontiguousarray(vf, dtype=np.float64)
    out = np.empty((len(xf) + 1) // 2, dtype=np.float64)
    lib.orc_line_restrict(len(xf), _dp(xf), _dp(vf), _dp(out))
    return out


def line_mass_solve(x, f):
    """z with M z = f (Thomas algorithm)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    z = np.empty_like(f)
    rc = lib.orc_line_mass_solve(len(f), _dp(x), _dp(f), _dp(z))
    if rc != 0:
        raise MemoryError("line solve allocation failed")
    return z
