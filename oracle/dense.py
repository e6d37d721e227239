"""Dense brute-force statement of the decomposition for tiny grids.

TEST INFRASTRUCTURE ONLY.  It shares nothing with ``mgard_oracle.c``: no
level recursion, no tridiagonal solve, no stencils.  It states the method
(Section II-A, Eq. 1-2) through global L2 projections:

* V_l is the space of continuous piecewise-multilinear functions on the
  nested node set N_l (Table 1); its basis is the tensor-product hat
  functions.
* Q_l u is the L2 projection of the piecewise-multilinear function u (nodal
  values on the finest grid) onto V_l: with G_l the Gram matrix of V_l and
  B_l the nodal values of the V_l basis on the finest grid,
  G_l q_l = B_l^T G_L u.
* The level-l coefficients are (I - Pi_{l-1}) Q_l u on N_l \\ N_{l-1}
  (Eq. 1); the coarsest nodes keep Q_0 u (Fig. 3 in-place layout).
* With a level count per dimension (``levels``), dimension k's node set
  stops thinning after levels[k] steps from the finest level; the spaces
  stay nested tensor products and everything above applies unchanged.

Gram matrices come from 2-point Gauss-Legendre quadrature of products of hat
functions on each element (exact for these quadratics); hat-function values
come from ``numpy.interp``.  Everything is dense and Kronecker-structured, so
keep grids to about a thousand nodes.
"""
from __future__ import annotations

import numpy as np


def level_index(n: int, L: int, l: int, Lk: int | None = None) -> np.ndarray:
    """Finest-grid indices of the level-l nodes of a dimension with n nodes
    (with Lk: a dimension that stops coarsening after Lk steps)."""
    step = L - l if Lk is None else min(L - l, Lk)
    return np.arange(0, n, 1 << step)


def _indices(coords, L, l, levels):
    return [level_index(len(x), L, l, None if levels is None else levels[k])
            for k, x in enumerate(coords)]


def gram_1d(x: np.ndarray) -> np.ndarray:
    """G_ij = integral of phi_i phi_j over [x_0, x_{n-1}] (hat functions on x)."""
    n = len(x)
    G = np.zeros((n, n))
    gp = np.array([-1.0, 1.0]) / np.sqrt(3.0)  # Gauss points on [-1, 1], weights 1
    for e in range(n - 1):
        a, b = x[e], x[e + 1]
        for t in gp:
            xi = 0.5 * (a + b) + 0.5 * (b - a) * t
            w = 0.5 * (b - a)
            phi = np.array([(b - xi) / (b - a), (xi - a) / (b - a)])
            G[e:e + 2, e:e + 2] += w * np.outer(phi, phi)
    return G


def hat_values(x_fine: np.ndarray, x_coarse: np.ndarray) -> np.ndarray:
    """B[j, i] = phi_i^coarse(x_fine[j]) for the hat functions on x_coarse."""
    B = np.zeros((len(x_fine), len(x_coarse)))
    for i in range(len(x_coarse)):
        e = np.zeros(len(x_coarse))
        e[i] = 1.0
        B[:, i] = np.interp(x_fine, x_coarse, e)
    return B


def _kron(mats):
    out = np.ones((1, 1))
    for m in mats:
        out = np.kron(out, m)
    return out


def projection(u: np.ndarray, coords, L: int, l: int, levels=None) -> np.ndarray:
    """Nodal values of Q_l u on N_l (array of the level-l shape)."""
    G_L = _kron([gram_1d(x) for x in coords])
    idx = _indices(coords, L, l, levels)
    B = _kron([hat_values(x, x[i]) for x, i in zip(coords, idx)])
    G_l = _kron([gram_1d(x[i]) for x, i in zip(coords, idx)])
    rhs = B.T @ (G_L @ u.reshape(-1))
    q = np.linalg.solve(G_l, rhs)
    return q.reshape([len(i) for i in idx])


def interpolate_from_coarse(q_l: np.ndarray, coords, L: int, l: int, levels=None) -> np.ndarray:
    """Pi_{l-1} q_l on N_l: multilinear interpolant of the N_{l-1} values."""
    idx_f = _indices(coords, L, l, levels)
    idx_c = _indices(coords, L, l - 1, levels)
    Bs = [hat_values(x[f], x[c]) for x, f, c in zip(coords, idx_f, idx_c)]
    coarse = q_l[tuple(np.ix_(*[np.searchsorted(f, c) for f, c in zip(idx_f, idx_c)]))]
    return (_kron(Bs) @ coarse.reshape(-1)).reshape(q_l.shape)


def decompose(u: np.ndarray, coords, L: int, levels=None) -> np.ndarray:
    """Full in-place decomposition array built from global projections
    (``levels``: per-dimension level counts, L their maximum)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    for l in range(L, 0, -1):
        q = projection(u, coords, L, l, levels)
        c = q - interpolate_from_coarse(q, coords, L, l, levels)
        idx = _indices(coords, L, l, levels)
        idx_c = _indices(coords, L, l - 1, levels)
        sub = out[np.ix_(*idx)]
        odd = np.zeros(q.shape, dtype=bool)
        for k in range(u.ndim):
            shp = [1] * u.ndim
            shp[k] = q.shape[k]
            odd = odd | (~np.isin(idx[k], idx_c[k])).reshape(shp)
        sub[odd] = c[odd]
        out[np.ix_(*idx)] = sub
    idx0 = _indices(coords, L, 0, levels)
    out[np.ix_(*idx0)] = projection(u, coords, L, 0, levels)
    return out
