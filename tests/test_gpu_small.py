"""The single-block coarse-level kernel against the FP64 oracle and against
the tiled per-level kernels (plan tuning parameter 3 switches between them;
parameter 4 keeps the cooperative kernel out, so that these plans take the
single-block kernel wherever it applies).

Shapes cover the three ways the kernel is entered: the whole field fits
(it runs every level on the user array), the field is large and the kernel
takes over at a coarse compact array, and the FP32 field with FP64 coarse
arrays (mixed precision), where the shared-memory array is in FP64.
Tolerances (max relative error over the array): 1e-12 FP64, 1e-5 FP32/mixed.
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
    ((33, 33, 33), "f32", False),       # whole field in one block
    ((17, 17, 17), "f64", False),
    ((65, 65, 65), "f32", False),       # tiled finest level, then the block
    ((65, 33, 129), "f64", True),
    ((33, 65, 33), "f32_mixed", False),
    ((129, 129), "f32", False),         # 2D: whole field
    ((257, 257), "f64", True),
    ((257,), "f32", False),             # 1D
    ((1025,), "f64", True),
]


def _field(shape, dtype, seed):
    npdt = np.float64 if dtype == "f64" else np.float32
    return synth.sinusoid_field(shape, 8, seed=seed, dtype=npdt)


@pytest.mark.parametrize("shape,dtype,nonuniform", CASES)
def test_small_path_matches_oracle_and_tiled(shape, dtype, nonuniform):
    mg = _mg()
    coords = _rand_coords(shape, 31) if nonuniform else None
    u = _field(shape, dtype, 30)
    plan = mg.Plan(shape, coords=coords, dtype=dtype)
    plan.tune(0, 4, 1)
    tiled = mg.Plan(shape, coords=coords, dtype=dtype)
    tiled.tune(0, 3, 1)
    assert mg.mgard_plan_get_tune(plan.handle, 0, 3) == 0
    assert mg.mgard_plan_get_tune(tiled.handle, 0, 3) == 1
    assert plan.launches() < tiled.launches()
    want = oracle.decompose(u.astype(np.float64), coords=coords)
    a = torch.from_numpy(u).cuda()
    b = a.clone()
    plan.decompose(a)
    tiled.decompose(b)
    torch.cuda.synchronize()
    ga, gb = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
    assert _relerr(ga, want) <= TOL[dtype]
    assert _relerr(gb, want) <= TOL[dtype]
    # recomposition of the oracle's coefficients
    c = torch.from_numpy(want.astype(u.dtype)).cuda()
    plan.recompose(c)
    torch.cuda.synchronize()
    back = oracle.recompose(want, coords=coords)
    assert _relerr(c.cpu().numpy().astype(np.float64), back) <= TOL[dtype]


@pytest.mark.parametrize("shape,dtype", [((33, 33, 33), "f32"), ((65, 65, 65), "f64"), ((129, 129), "f32")])
def test_small_path_round_trip(shape, dtype):
    mg = _mg()
    u = _field(shape, dtype, 32)
    plan = mg.Plan(shape, dtype=dtype)
    plan.tune(0, 4, 1)
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    plan.recompose(t)
    torch.cuda.synchronize()
    assert _relerr(t.cpu().numpy().astype(np.float64), u.astype(np.float64)) <= TOL[dtype]


def test_small_switch_rejects_bad_value():
    mg = _mg()
    plan = mg.Plan((33, 33, 33), dtype="f32")
    with pytest.raises(mg.MgardError):
        plan.tune(0, 3, 2)
