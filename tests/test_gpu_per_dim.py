"""Per-dimension level counts on the GPU (the persistent kernel runs such
plans): each dimension coarsens in its own first L_k steps and then keeps
its nodes.  Parity with the FP64 oracle's per-dimension maps in both
directions (FP32 1e-5, FP64 1e-12, the mixed scheme 1e-5) on shapes where
the first, the middle and the last dimension stop early, 2D fields stopping
along rows or columns, partial level vectors, graded coordinates and uneven
sides; equal counts give the plain plan; calls a per-dimension plan does
not support fail cleanly.
"""
import numpy as np
import pytest

import oracle
from paper_2007_04457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-12, "f32_mixed": 1e-5}


def _mg():
    from paper_2007_04457_gb300 import mgard
    return mgard


def _np(dtype):
    return np.float64 if dtype == "f64" else np.float32


def _coords(shape, seed):
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
    # shape, per-dimension levels (None = each dimension's maximum), graded
    ((9, 65, 33), None, False),          # dim 0 stops after 3 levels, dim 2 after 5
    ((65, 9, 33), None, True),           # dim 1 stops first: levels run by rows
    ((33, 65, 5), None, False),          # the contiguous dim stops after 2 levels
    ((17, 33, 65), (2, 4, 3), True),     # partial counts, every dim different
    ((129, 17), None, False),            # 2D, the column dim stops first
    ((17, 257), (4, 6), True),           # 2D, the row dim stops first
    ((33, 33, 9), (5, 1, 3), False),     # dim 1 stops after one level
    ((257,), None, False),               # 1D (a single dimension)
    ((9, 6), (3, 0), False),             # a dimension that never coarsens (even size)
    ((13, 9), (2, 3), True),
    ((17, 5, 9), (4, 2, 3), False),
    ((5, 9, 17), (2, 3, 4), True),
]


@pytest.mark.parametrize("dtype", ["f32", "f64", "f32_mixed"])
@pytest.mark.parametrize("shape,levels,graded", CASES)
def test_per_dim_plan_matches_oracle(shape, levels, graded, dtype):
    mg = _mg()
    coords = _coords(shape, 7) if graded else None
    lv = oracle.dim_levels(shape) if levels is None else levels
    plan = mg.Plan(shape, coords=coords, dtype=dtype, dim_levels=levels if levels is not None else "max")
    assert plan.levels == max(lv)
    u = synth.sinusoid_field(shape, 12 if len(shape) == 3 else 8, seed=13).astype(_np(dtype))
    t = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    want = oracle.decompose_per_dim(u.astype(np.float64), lv, coords)
    got = t.cpu().numpy().astype(np.float64)
    assert _relerr(got, want) <= TOL[dtype], _relerr(got, want)
    c = want.astype(_np(dtype))
    t2 = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    plan.recompose(t2)
    torch.cuda.synchronize()
    want_r = oracle.recompose_per_dim(c.astype(np.float64), lv, coords)
    assert _relerr(t2.cpu().numpy().astype(np.float64), want_r) <= TOL[dtype]
    # round trip on the device
    plan.recompose(t)
    torch.cuda.synchronize()
    assert _relerr(t.cpu().numpy().astype(np.float64), u.astype(np.float64)) <= 10 * TOL[dtype]


def test_equal_counts_give_the_plain_plan():
    mg = _mg()
    shape = (33, 33, 65)
    per = mg.Plan(shape, dtype="f32", dim_levels=(4, 4, 4))
    plain = mg.Plan(shape, nlevels=4, dtype="f32")
    assert per.levels == plain.levels == 4
    assert per.launches() == plain.launches()
    u = synth.sinusoid_field(shape, 12, seed=3, dtype=np.float32)
    a = torch.from_numpy(u).cuda()
    b = a.clone()
    per.decompose(a)
    plain.decompose(b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_per_dim_plan_refuses_what_it_does_not_support():
    mg = _mg()
    plan = mg.Plan((9, 65, 33), dtype="f32", dim_levels="max")
    assert plan.launches() == 1
    t = torch.zeros(plan.shape, device="cuda")
    with pytest.raises(mg.MgardError):
        plan.decompose_adjoint(t)
    with pytest.raises(mg.MgardError):
        plan.tune(0, 3, 1)
    with pytest.raises(mg.MgardError):   # rows longer than the persistent kernel takes
        mg.Plan((5, 2049), dtype="f32", dim_levels="max")
    with pytest.raises(mg.MgardError):   # more levels than the dimension allows
        mg.Plan((9, 65), dtype="f32", dim_levels=(4, 2))
