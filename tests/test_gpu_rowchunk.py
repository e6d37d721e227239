"""GPU parity of the row-chunk level kernels (one warp per row segment in
aligned 16-byte words, the restriction fused with the dim-2 solve where a
row is one segment) against the FP64 oracle, and against the tile / strip
kernels they replace (tuning param 7: 0 = all row-chunk kernels, 3 = none).

Every level runs the per-level kernels here (tuning param 3 = 1), so the
row-chunk kernels take every level whose rows they fit, not only the ones
above the single launch of the coarse end.  Shapes cover one and several
segments per row (512- and 256-column segments), 2D and 3D, FP32, FP64 and
the mixed scheme, uniform and graded coordinates, partial level counts,
levels the kernels do not take between ones they do, and a user array that
is not 16-byte aligned (its level falls back to the other kernels).
"""
import numpy as np
import pytest

import oracle
from paper_2007_04457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32_mixed": 1e-5}


def _mg():
    from paper_2007_04457_gb300 import mgard
    return mgard


def _np(dtype):
    return np.float64 if dtype == "f64" else np.float32


def _rand_coords(shape, seed):
    rng = np.random.default_rng(seed)
    out = []
    for n in shape:
        h = rng.uniform(0.5, 1.0, n - 1)
        x = np.concatenate([[0.0], np.cumsum(h)])
        out.append(x / x[-1])
    return out


def _relerr(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


CASES = [
    # shape, dtype, nlevels, nonuniform, restriction segment width of level 0
    ((9, 17, 257), "f32", -1, False, 256),        # one 256-column segment: fused x solve
    ((9, 9, 513), "f32", -1, False, 512),         # one 512-column segment
    ((5, 17, 1025), "f32", -1, True, 512),        # two segments per row, graded grid
    ((17, 17, 513), "f64", -1, False, 256),       # FP64: two 256-column segments
    ((9, 25, 257), "f64", -1, True, 256),         # level 1 (n1 = 13) not a row-chunk level
    ((9, 17, 513), "f32_mixed", -1, False, 512),
    ((9, 33, 1025), "f32_mixed", 2, True, 512),   # partial level count
    ((33, 513), "f32", -1, False, 512),           # 2D
    ((17, 1025), "f64", -1, True, 256),           # 2D, four segments
    ((65, 257), "f32_mixed", -1, False, 256),     # 2D mixed
]


def _plan(mg, shape, dtype, nlevels, coords, rc):
    plan = mg.Plan(shape, nlevels=nlevels, coords=coords, dtype=dtype)
    plan.tune(0, 3, 1)          # every level with the per-level kernels
    plan.tune(0, 7, 0 if rc else 3)
    return plan


def _run(plan, fn, host, dtype, offset=0):
    n = host.size
    buf = torch.empty(n + offset, dtype=plan.torch_dtype, device="cuda")
    t = buf[offset:].view(host.shape)
    t.copy_(torch.from_numpy(np.ascontiguousarray(host.astype(_np(dtype)))))
    getattr(plan, fn)(t)
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("shape,dtype,nlevels,nonuniform,width", CASES)
def test_rowchunk_levels_match_oracle(shape, dtype, nlevels, nonuniform, width):
    mg = _mg()
    coords = _rand_coords(shape, 11) if nonuniform else None
    u = synth.sinusoid_field(shape, 12 if len(shape) == 3 else 8, seed=6).astype(_np(dtype))
    plan = _plan(mg, shape, dtype, nlevels, coords, True)
    assert mg.mgard_plan_get_tune(plan.handle, 0, 8) == width
    got = _run(plan, "decompose", u, dtype)
    want = oracle.decompose(u.astype(np.float64), nlevels=plan.levels, coords=coords)
    assert _relerr(got, want) <= TOL[dtype], _relerr(got, want)
    # recomposition of the oracle's coefficients
    c = want.astype(_np(dtype))
    got_r = _run(plan, "recompose", c, dtype)
    want_r = oracle.recompose(c.astype(np.float64), nlevels=plan.levels, coords=coords)
    assert _relerr(got_r, want_r) <= TOL[dtype], _relerr(got_r, want_r)
    # the tile / strip kernels on the same input agree to rounding
    plan_off = _plan(mg, shape, dtype, nlevels, coords, False)
    other = _run(plan_off, "decompose", u, dtype)
    assert _relerr(got, other) <= 2 * TOL[dtype]
    plan.close()
    plan_off.close()


@pytest.mark.parametrize("shape,dtype", [((9, 17, 513), "f32"), ((17, 257), "f32_mixed")])
def test_unaligned_user_array_falls_back(shape, dtype):
    """A user array 4 bytes off a 16-byte boundary: level 0 takes the other
    kernels (level 1 works on the aligned workspace with row-chunk kernels
    where it fits); the result still matches the oracle."""
    mg = _mg()
    u = synth.sinusoid_field(shape, 12, seed=9).astype(_np(dtype))
    plan = _plan(mg, shape, dtype, -1, None, True)
    got = _run(plan, "decompose", u, dtype, offset=1)
    want = oracle.decompose(u.astype(np.float64), nlevels=plan.levels)
    assert _relerr(got, want) <= TOL[dtype]
    got_r = _run(plan, "recompose", want.astype(_np(dtype)), dtype, offset=1)
    assert _relerr(got_r, u.astype(np.float64)) <= 10 * TOL[dtype]


@pytest.mark.parametrize("zreq", [1, 3, 16, 64])
@pytest.mark.parametrize("dtype", ["f32", "f64", "f32_mixed"])
def test_rowchunk_long_plane_chunks(zreq, dtype):
    """Work items that stream many planes (tuning param 9), so that every
    prefetched row of a warp's ring is a live row of the item: parity with
    the oracle in both directions on a 3D grid with 129 planes."""
    mg = _mg()
    shape = (129, 17, 257)
    u = synth.sinusoid_field(shape, 12, seed=12).astype(_np(dtype))
    plan = _plan(mg, shape, dtype, 2, None, True)
    plan.tune(0, 9, zreq)
    got = _run(plan, "decompose", u, dtype)
    want = oracle.decompose(u.astype(np.float64), nlevels=plan.levels)
    assert _relerr(got, want) <= TOL[dtype], _relerr(got, want)
    got_r = _run(plan, "recompose", want.astype(_np(dtype)), dtype)
    want_r = oracle.recompose(want, nlevels=plan.levels)
    assert _relerr(got_r, want_r) <= TOL[dtype], _relerr(got_r, want_r)


def test_rowchunk_default_plan_round_trip_1025_rows():
    """The default plan (coarse end in one launch) of a 3D field with rows of
    1025 nodes, decomposed and recomposed twice in a row: parity with the
    oracle and a repeatable round trip."""
    mg = _mg()
    shape = (17, 33, 1025)
    u = synth.sinusoid_field(shape, 12, seed=10, dtype=np.float32)
    plan = mg.Plan(shape, dtype="f32")
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    first = t.cpu().numpy().astype(np.float64)
    want = oracle.decompose(u.astype(np.float64), nlevels=plan.levels)
    assert _relerr(first, want) <= 1e-5
    plan.recompose(t)
    plan.decompose(t)
    torch.cuda.synchronize()
    assert _relerr(t.cpu().numpy().astype(np.float64), want) <= 1e-5
