"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics (no GPU).  Each test names what it pins.

Section II-A (Eq. 1-2) defines the decomposition; the oracle follows it level
by level.  These tests check it against an independent dense statement, closed
forms, invariants and the hand-worked 1D example of Fig. 2.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_coords(rng, shape):
    out = []
    for n in shape:
        inner = np.sort(rng.uniform(0.0, 1.0, n - 2))
        out.append(np.concatenate([[0.0], inner, [1.0]]))
    return out


def _relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ---------------------------------------------------------------- worked example

def test_worked_example_1d_fig2():
    """Fig. 2 function y = x^2-5x+6 on x = 0..4, two levels, worked by hand."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "worked_example_1d.txt"))
            if l.strip() and not l.startswith("#")]
    x, u, want = (np.array([float(v) for v in r]) for r in rows)
    got = oracle.decompose(u, coords=[x])
    assert np.array_equal(got, want)
    # the Thomas divisions round (1/3-type pivots), so the way back is exact
    # only to FP64 rounding
    np.testing.assert_allclose(oracle.recompose(want, coords=[x]), u, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("shape", [(17,), (9, 17), (9, 5, 17)])
def test_quadratic_closed_form(shape):
    """u = sum_k x_k^2: the finest coefficient at a node odd in the set S of
    dimensions is -sum_{k in S} h_k^2 (multilinear interpolation of x^2)."""
    coords = [np.arange(n) * (0.5 + k) for k, n in enumerate(shape)]
    h = [c[1] - c[0] for c in coords]
    u = np.zeros(shape)
    for k, c in enumerate(coords):
        s = [1] * len(shape)
        s[k] = shape[k]
        u = u + (c ** 2).reshape(s)
    out = oracle.decompose(u, nlevels=1, coords=coords)
    want = np.zeros(shape)
    any_odd = np.zeros(shape, dtype=bool)
    for k, n in enumerate(shape):
        s = [1] * len(shape)
        s[k] = n
        odd_k = (np.arange(n) % 2 == 1).reshape(s)
        want = want - np.where(odd_k, h[k] ** 2, 0.0)
        any_odd = any_odd | odd_k
    np.testing.assert_allclose(out[any_odd], want[any_odd], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("shape,l0", [((33,), 2), ((17, 9), 1), ((9, 9, 17), 1), ((17, 17, 9), 0)])
def test_piecewise_multilinear_input_has_zero_finer_coefficients(shape, l0):
    """u piecewise multilinear on N_{l0}: every coefficient above level l0 is
    exactly zero and the N_{l0} values come out as the l0-level
    decomposition of the coarse data (dyadic values keep it exact)."""
    rng = np.random.default_rng(3)
    L = oracle.max_levels(shape)
    stride = 1 << (L - l0)
    cshape = tuple((n - 1) // stride + 1 for n in shape)
    coarse = rng.integers(-8, 9, size=cshape).astype(np.float64)
    # exact dyadic prolongation on the uniform grid, one dimension at a time
    u = coarse
    for k in range(len(shape)):
        for _ in range(L - l0):
            n = u.shape[k]
            new_shape = list(u.shape)
            new_shape[k] = 2 * n - 1
            v = np.zeros(new_shape)
            sl = [slice(None)] * len(shape)
            sl[k] = slice(0, None, 2)
            v[tuple(sl)] = u
            a = [slice(None)] * len(shape)
            b = [slice(None)] * len(shape)
            o = [slice(None)] * len(shape)
            a[k] = slice(0, -1)
            b[k] = slice(1, None)
            o[k] = slice(1, None, 2)
            v[tuple(o)] = 0.5 * (u[tuple(a)] + u[tuple(b)])
            u = v
    assert u.shape == shape
    out = oracle.decompose(u, nlevels=L)
    idx = np.ix_(*[np.arange(0, n, stride) for n in shape])
    rest = np.ones(shape, dtype=bool)
    rest[idx] = False
    assert np.all(out[rest] == 0.0)
    want = oracle.decompose(coarse, nlevels=l0) if l0 > 0 else coarse
    assert np.array_equal(out[idx], want)


def test_constant_input():
    """A constant field: coarsest values equal the constant, all coefficients 0."""
    u = np.full((9, 17, 33), 2.5)
    out = oracle.decompose(u)
    stride = 1 << oracle.max_levels(u.shape)
    idx = np.ix_(*[np.arange(0, n, stride) for n in u.shape])
    assert np.all(out[idx] == 2.5)
    rest = np.ones(u.shape, dtype=bool)
    rest[idx] = False
    assert np.all(out[rest] == 0.0)


# ---------------------------------------------------------------- dense brute force

@pytest.mark.parametrize("shape", [(33,), (17, 9), (9, 9, 9), (5, 9, 17)])
@pytest.mark.parametrize("uniform", [True, False])
@pytest.mark.parametrize("partial", [False, True])
def test_matches_dense_projections(shape, uniform, partial):
    """Whole decomposition equals the global-projection statement of Eq. 1:
    level-l coefficients (I - Pi_{l-1}) Q_l u, coarsest values Q_0 u, with Q_l
    from dense Gram systems (no recursion, no Thomas, no stencils)."""
    rng = np.random.default_rng(11)
    coords = ([oracle.uniform_coords(n) for n in shape] if uniform
              else _rand_coords(rng, shape))
    L = oracle.max_levels(shape)
    if partial:
        L = max(1, L - 1)
    u = rng.standard_normal(shape)
    got = oracle.decompose(u, nlevels=L, coords=coords)
    want = dense.decompose(u, coords, L)
    assert _relmax(got, want) < 1e-12


@pytest.mark.parametrize("shape", [(33,), (9, 17), (9, 9, 9)])
def test_projection_orthogonality(shape):
    """u - Q_l u is L2-orthogonal to V_l at every level (Section II-A-2)."""
    rng = np.random.default_rng(5)
    coords = _rand_coords(rng, shape)
    L = oracle.max_levels(shape)
    u = rng.standard_normal(shape)
    G_L = dense._kron([dense.gram_1d(x) for x in coords])
    for l in range(L - 1, -1, -1):
        part = oracle.decompose(u, nlevels=L - l, coords=coords)
        idx = [dense.level_index(len(x), L, l) for x in coords]
        q = part[np.ix_(*idx)]
        B = dense._kron([dense.hat_values(x, x[i]) for x, i in zip(coords, idx)])
        resid = B.T @ (G_L @ (u.reshape(-1) - B @ q.reshape(-1)))
        scale = np.abs(B.T @ (G_L @ u.reshape(-1))).max()
        assert np.abs(resid).max() < 1e-12 * scale


def test_separable_product_is_outer_product():
    """For u = a(x) b(y) c(z), Q_l is a tensor product, so the N_l values of
    the 3D decomposition are the outer product of the 1D ones."""
    rng = np.random.default_rng(8)
    shape = (9, 17, 33)
    coords = _rand_coords(rng, shape)
    fac = [rng.standard_normal(n) for n in shape]
    u = np.einsum("i,j,k->ijk", *fac)
    L = oracle.max_levels(shape)
    for k in range(1, L + 1):
        full = oracle.decompose(u, nlevels=k, coords=coords)
        ones = [oracle.decompose(f, nlevels=k, coords=[c]) for f, c in zip(fac, coords)]
        stride = 1 << k
        idx = [np.arange(0, n, stride) for n in shape]
        want = np.einsum("i,j,k->ijk", *[o[i] for o, i in zip(ones, idx)])
        assert _relmax(full[np.ix_(*idx)], want) < 1e-12


# ---------------------------------------------------------------- invariants

def test_linearity():
    rng = np.random.default_rng(2)
    shape = (17, 9, 17)
    coords = _rand_coords(rng, shape)
    a, b = rng.standard_normal(shape), rng.standard_normal(shape)
    lhs = oracle.decompose(2.5 * a - 0.75 * b, coords=coords)
    rhs = 2.5 * oracle.decompose(a, coords=coords) - 0.75 * oracle.decompose(b, coords=coords)
    assert _relmax(lhs, rhs) < 1e-13


def test_coordinate_scaling_and_shift_invariance():
    """Scaling or shifting one axis rescales M_l and M_{l-1} alike and leaves
    interpolation weights unchanged, so the result is invariant."""
    rng = np.random.default_rng(4)
    shape = (9, 17, 33)
    coords = _rand_coords(rng, shape)
    u = rng.standard_normal(shape)
    base = oracle.decompose(u, coords=coords)
    moved = [coords[0] * 3.7 + 1.0, coords[1], coords[2] * 0.01]
    assert _relmax(oracle.decompose(u, coords=moved), base) < 1e-12


@pytest.mark.parametrize("shape", [(65,), (33, 17), (17, 9, 33), (9, 9, 5)])
@pytest.mark.parametrize("uniform", [True, False])
def test_round_trip(shape, uniform):
    """recompose(decompose(u)) == u to FP64 rounding (Section II-A: recomposition
    runs the same stages in reverse)."""
    rng = np.random.default_rng(6)
    coords = ([oracle.uniform_coords(n) for n in shape] if uniform
              else _rand_coords(rng, shape))
    u = rng.standard_normal(shape)
    for L in range(0, oracle.max_levels(shape) + 1):
        back = oracle.recompose(oracle.decompose(u, nlevels=L, coords=coords),
                                nlevels=L, coords=coords)
        assert _relmax(back, u) < 1e-14 * max(1, L)


# ---------------------------------------------------------------- adjoints

def _dense_map(fn, shape, coords):
    n = int(np.prod(shape))
    D = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        D[:, i] = fn(e.reshape(shape), coords=coords).reshape(-1)
    return D


@pytest.mark.parametrize("shape", [(17,), (9, 5), (5, 5, 9)])
def test_adjoints_are_dense_transposes(shape):
    rng = np.random.default_rng(9)
    coords = _rand_coords(rng, shape)
    D = _dense_map(oracle.decompose, shape, coords)
    Dt = _dense_map(oracle.decompose_adjoint, shape, coords)
    assert np.abs(D.T - Dt).max() < 1e-13 * np.abs(D).max()
    R = _dense_map(oracle.recompose, shape, coords)
    Rt = _dense_map(oracle.recompose_adjoint, shape, coords)
    assert np.abs(R.T - Rt).max() < 1e-13 * np.abs(R).max()
    assert np.abs(R @ D - np.eye(D.shape[0])).max() < 1e-13


def test_adjoint_dot_products():
    """|<Dx, y> - <x, D^T y>| <= 1e-12 ||Dx|| ||y|| on a 17^3 grid."""
    rng = np.random.default_rng(10)
    shape = (17, 17, 17)
    coords = _rand_coords(rng, shape)
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    for fwd, adj in ((oracle.decompose, oracle.decompose_adjoint),
                     (oracle.recompose, oracle.recompose_adjoint)):
        Dx = fwd(x, coords=coords)
        lhs = np.vdot(Dx, y)
        rhs = np.vdot(x, adj(y, coords=coords))
        assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Dx) * np.linalg.norm(y)
    back = oracle.recompose_adjoint(oracle.decompose_adjoint(y, coords=coords), coords=coords)
    assert _relmax(back, y) < 1e-13


# ---------------------------------------------------------------- line operators

def _line_matrix(fn, n_in, n_out, *args):
    A = np.zeros((n_out, n_in))
    for i in range(n_in):
        e = np.zeros(n_in)
        e[i] = 1.0
        A[:, i] = fn(*args, e)
    return A


def test_mass_matrix_is_six_times_gram():
    """The oracle's M is 6x the L2 Gram matrix of the hat functions (exact
    Gauss quadrature), Section III-A-2."""
    rng = np.random.default_rng(12)
    x = _rand_coords(rng, (23,))[0]
    M = _line_matrix(oracle.line_mass, 23, 23, x)
    assert np.abs(M - 6.0 * dense.gram_1d(x)).max() < 1e-14


def test_galerkin_identity_and_transfer():
    """P^T M_l P = M_{l-1} (nested hat functions); R = P^T."""
    rng = np.random.default_rng(13)
    xf = _rand_coords(rng, (33,))[0]
    xc = xf[::2]
    P = _line_matrix(oracle.line_prolong, 17, 33, xf)
    R = _line_matrix(oracle.line_restrict, 33, 17, xf)
    Mf = _line_matrix(oracle.line_mass, 33, 33, xf)
    Mc = _line_matrix(oracle.line_mass, 17, 17, xc)
    assert np.abs(R - P.T).max() == 0.0
    assert np.abs(P.T @ Mf @ P - Mc).max() < 1e-14 * np.abs(Mc).max()


def test_prolongation_reproduces_linear_functions():
    """P interpolates exactly: linear data on N_{l-1} stays linear on N_l."""
    rng = np.random.default_rng(14)
    xf = _rand_coords(rng, (41,))[0]
    out = oracle.line_prolong(xf, 3.0 * xf[::2] - 1.25)
    np.testing.assert_allclose(out, 3.0 * xf - 1.25, rtol=0, atol=1e-14)
    np.testing.assert_allclose(out, dense.hat_values(xf, xf[::2]) @ (3.0 * xf[::2] - 1.25),
                               rtol=0, atol=1e-14)


@pytest.mark.parametrize("n", [2, 3, 17, 257])
def test_thomas_matches_dense_solve(n):
    rng = np.random.default_rng(15)
    x = _rand_coords(rng, (n,))[0] if n > 2 else np.array([0.0, 0.7])
    f = rng.standard_normal(n)
    M = _line_matrix(oracle.line_mass, n, n, x)
    z = oracle.line_mass_solve(x, f)
    np.testing.assert_allclose(z, np.linalg.solve(M, f), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- coefficient classes

def _on_finest(q, coords, L, k):
    """Finest-grid nodal values of the V_k function with nodal values q on N_k
    (tensor product of 1D hat-function evaluations)."""
    B = np.ones((1, 1))
    for x in coords:
        B = np.kron(B, dense.hat_values(x, x[dense.level_index(len(x), L, k)]))
    return (B @ q.reshape(-1)).reshape([len(x) for x in coords])


@pytest.mark.parametrize("shape", [(33,), (17, 9), (9, 9, 9), (5, 9, 17)])
@pytest.mark.parametrize("uniform", [True, False])
def test_classes_give_projections(shape, uniform):
    """Keeping the first k+1 classes rebuilds Q_k u, the L2 projection onto
    V_k (u = Q_0 u + sum_l (Q_l - Q_{l-1}) u, each class one term), from
    dense Gram systems; all L+1 classes give u back."""
    rng = np.random.default_rng(21)
    coords = ([oracle.uniform_coords(n) for n in shape] if uniform
              else _rand_coords(rng, shape))
    L = oracle.max_levels(shape)
    u = rng.standard_normal(shape)
    dec = oracle.decompose(u, coords=coords)
    for nc in range(1, L + 2):
        got = oracle.recompose_classes(dec, nc, coords=coords)
        want = _on_finest(dense.projection(u, coords, L, nc - 1), coords, L, nc - 1)
        assert _relmax(got, want) < 1e-11, nc


@pytest.mark.parametrize("shape,k", [((33,), 2), ((17, 9), 1), ((9, 9, 17), 2), ((17, 17, 9), 0)])
def test_classes_reproduce_level_k_functions(shape, k):
    """A function of V_k is its own projection: its first k+1 classes
    rebuild it, non-uniform spacing included."""
    rng = np.random.default_rng(5)
    coords = _rand_coords(rng, shape)
    L = oracle.max_levels(shape)
    q = rng.standard_normal([len(dense.level_index(n, L, k)) for n in shape])
    u = _on_finest(q, coords, L, k)
    got = oracle.recompose_classes(oracle.decompose(u, coords=coords), k + 1, coords=coords)
    assert _relmax(got, u) < 1e-12


def test_classes_error_is_monotone():
    """V_0 in V_1 in ... in V_L, and Q_k is the best approximation in V_k
    in the L2 norm, so the L2 error of the rebuilt field never grows with
    the number of classes kept and reaches zero with all of them."""
    rng = np.random.default_rng(8)
    shape = (9, 17, 9)
    coords = _rand_coords(rng, shape)
    L = oracle.max_levels(shape)
    G = np.ones((1, 1))
    for x in coords:
        G = np.kron(G, dense.gram_1d(x))
    u = rng.standard_normal(shape)
    dec = oracle.decompose(u, coords=coords)
    errs = []
    for nc in range(1, L + 2):
        e = (u - oracle.recompose_classes(dec, nc, coords=coords)).reshape(-1)
        errs.append(float(e @ G @ e))
    assert all(b <= a * (1 + 1e-12) + 1e-24 for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-24 and errs[0] > 1e-3


def test_classes_worked_example_1d():
    """Fig. 2 example rebuilt from its first 1, 2 and 3 classes, worked by
    hand (tests/golden/classes_1d.txt)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "classes_1d.txt"))
            if l.strip() and not l.startswith("#")]
    x, dec, *want = (np.array([float(v) for v in r]) for r in rows)
    for nc, w in enumerate(want, start=1):
        np.testing.assert_allclose(oracle.recompose_classes(dec, nc, coords=[x]), w, rtol=0, atol=1e-14)


def test_classes_argument_range():
    u = np.zeros((9, 9))
    with pytest.raises(ValueError):
        oracle.recompose_classes(u, 0)
    with pytest.raises(ValueError):
        oracle.recompose_classes(u, oracle.max_levels(u.shape) + 2)


# ---------------------------------------------------------------- per-dimension level counts

PER_DIM = [((33, 5), (5, 2)), ((9, 33), (3, 5)), ((17, 5, 9), (4, 2, 3)),
           ((5, 9, 17), (2, 3, 4)), ((9, 6), (3, 0)), ((13, 9), (2, 3))]


def test_per_dim_default_levels():
    assert oracle.dim_levels((1025, 1025, 513)) == (10, 10, 9)
    assert oracle.dim_levels((17, 6)) == (4, 0)
    assert oracle.dim_levels((13,)) == (2,)     # 12 = 3 * 4
    assert oracle.dim_levels((2, 3)) == (0, 1)


@pytest.mark.parametrize("shape", [(33,), (9, 17), (17, 9, 33)])
def test_per_dim_equal_levels_is_the_plain_map(shape):
    """Every dimension with the same count L: the plain maps, bit for bit."""
    rng = np.random.default_rng(31)
    coords = _rand_coords(rng, shape)
    L = oracle.max_levels(shape)
    u = rng.standard_normal(shape)
    lv = (L,) * len(shape)
    assert np.array_equal(oracle.decompose_per_dim(u, lv, coords), oracle.decompose(u, L, coords))
    assert np.array_equal(oracle.recompose_per_dim(u, lv, coords), oracle.recompose(u, L, coords))
    assert np.array_equal(oracle.decompose_adjoint_per_dim(u, lv, coords),
                          oracle.decompose_adjoint(u, L, coords))


@pytest.mark.parametrize("shape,levels", PER_DIM)
@pytest.mark.parametrize("uniform", [True, False])
def test_per_dim_matches_dense_projections(shape, levels, uniform):
    """Unequal level counts against the global-projection statement on
    per-dimension nested node sets (no recursion, no Thomas, no stencils)."""
    rng = np.random.default_rng(12)
    coords = ([oracle.uniform_coords(n) for n in shape] if uniform
              else _rand_coords(rng, shape))
    u = rng.standard_normal(shape)
    got = oracle.decompose_per_dim(u, levels, coords)
    want = dense.decompose(u, coords, max(levels), levels)
    assert _relmax(got, want) < 1e-12


@pytest.mark.parametrize("shape,levels,axis", [((17, 6), (4, 0), 1), ((6, 33), (0, 5), 0)])
def test_per_dim_frozen_dimension_gives_independent_lines(shape, levels, axis):
    """A dimension that never coarsens contributes the identity: every line
    across it is decomposed on its own by the 1D map (mass matrix and its
    inverse cancel along the frozen dimension)."""
    rng = np.random.default_rng(4)
    coords = _rand_coords(rng, shape)
    u = rng.standard_normal(shape)
    got = oracle.decompose_per_dim(u, levels, coords)
    live = 1 - axis
    for j in range(shape[axis]):
        sl = (slice(None), j) if axis == 1 else (j, slice(None))
        want = oracle.decompose(u[sl], levels[live], [coords[live]])
        assert _relmax(got[sl], want) < 1e-12


def test_per_dim_frozen_dimension_in_3d_gives_independent_planes():
    shape, levels = (5, 6, 9), (2, 0, 3)
    rng = np.random.default_rng(6)
    coords = _rand_coords(rng, shape)
    u = rng.standard_normal(shape)
    got = oracle.decompose_per_dim(u, levels, coords)
    for j in range(shape[1]):
        want = dense.decompose(u[:, j, :], [coords[0], coords[2]], 3, (2, 3))
        assert _relmax(got[:, j, :], want) < 1e-12


@pytest.mark.parametrize("shape,levels", PER_DIM)
def test_per_dim_round_trip(shape, levels):
    rng = np.random.default_rng(13)
    coords = _rand_coords(rng, shape)
    u = rng.standard_normal(shape)
    back = oracle.recompose_per_dim(oracle.decompose_per_dim(u, levels, coords), levels, coords)
    assert _relmax(back, u) < 1e-13


@pytest.mark.parametrize("shape,levels", PER_DIM[:4])
def test_per_dim_adjoint_dot_products(shape, levels):
    """<D x, y> = <x, D^T y> for both maps."""
    rng = np.random.default_rng(14)
    coords = _rand_coords(rng, shape)
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    for fwd, adj in ((oracle.decompose_per_dim, oracle.decompose_adjoint_per_dim),
                     (oracle.recompose_per_dim, oracle.recompose_adjoint_per_dim)):
        dx = fwd(x, levels, coords)
        lhs = float(np.sum(dx * y))
        rhs = float(np.sum(x * adj(y, levels, coords)))
        assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(dx) * np.linalg.norm(y)


def test_per_dim_level_count_beyond_the_side_is_rejected():
    u = np.zeros((9, 6))
    with pytest.raises(ValueError):
        oracle.decompose_per_dim(u, (3, 1))     # 5 is not divisible by 2
    with pytest.raises(ValueError):
        oracle.decompose_per_dim(u, (3,))
