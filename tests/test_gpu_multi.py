"""The cooperative coarse-level kernel against the FP64 oracle, the
single-block kernel and the tiled per-level kernels.

A plan runs every level from the first whose array has sides <= 129 nodes in
one cooperative launch per direction: the whole grid works on each level
until the array has at most 1000 nodes, then one block finishes the rest in
shared memory.  Plan tuning parameter 4 switches back to the single-block
kernel, parameter 3 to the tiled kernels for every level; mgard_plan_get_tune
reports the first cooperative level as parameter 5.  Shapes cover the
kernel's entries: on the user array (level 0, also FP32 user data with FP64
levels), on a compact coarse array after tiled levels, 2D grids, anisotropic
and non-uniform grids.  Tolerances (max relative error): 1e-12 FP64, 1e-5
FP32 and mixed.
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


def _field(shape, dtype, seed):
    npdt = np.float64 if dtype == "f64" else np.float32
    return synth.sinusoid_field(shape, 8, seed=seed, dtype=npdt)


# shape, dtype, non-uniform coordinates, first cooperative level
CASES = [
    ((129, 129, 129), "f32", False, 0),
    ((129, 129, 129), "f64", True, 0),
    ((129, 129, 129), "f32_mixed", False, 0),
    ((65, 65, 65), "f64", False, 0),
    ((33, 33, 33), "f32", False, 0),
    ((257, 257, 257), "f32", False, 1),
    ((65, 129, 257), "f64", True, 1),
    ((257, 129, 129), "f32_mixed", True, 1),
    ((129, 129), "f64", False, 0),
    ((1025, 1025), "f32", False, 3),
    ((513, 257), "f64", True, 2),
]


@pytest.mark.parametrize("shape,dtype,nonuniform,coop", CASES)
def test_multi_matches_oracle_and_other_paths(shape, dtype, nonuniform, coop):
    mg = _mg()
    coords = _rand_coords(shape, 51) if nonuniform else None
    u = _field(shape, dtype, 50)
    plan = mg.Plan(shape, coords=coords, dtype=dtype)
    single = mg.Plan(shape, coords=coords, dtype=dtype)
    single.tune(0, 4, 1)
    tiled = mg.Plan(shape, coords=coords, dtype=dtype)
    tiled.tune(0, 3, 1)
    assert mg.mgard_plan_get_tune(plan.handle, 0, 5) == coop
    assert mg.mgard_plan_get_tune(single.handle, 0, 5) == -1
    assert mg.mgard_plan_get_tune(tiled.handle, 0, 5) == -1
    assert plan.launches() < tiled.launches()
    want = oracle.decompose(u.astype(np.float64), coords=coords)
    outs = []
    for p in (plan, single, tiled):
        a = torch.from_numpy(u).cuda()
        p.decompose(a)
        outs.append(a)
    torch.cuda.synchronize()
    for a in outs:
        assert _relerr(a.cpu().numpy().astype(np.float64), want) <= TOL[dtype]
    # recomposition of the oracle's coefficients
    back = oracle.recompose(want, coords=coords)
    c = torch.from_numpy(want.astype(u.dtype)).cuda()
    plan.recompose(c)
    torch.cuda.synchronize()
    assert _relerr(c.cpu().numpy().astype(np.float64), back) <= TOL[dtype]


@pytest.mark.parametrize("shape,dtype", [((129, 129, 129), "f32"), ((257, 257, 257), "f64"), ((1025, 1025), "f32_mixed")])
def test_multi_round_trip_and_repeatable(shape, dtype):
    mg = _mg()
    u = _field(shape, dtype, 52)
    plan = mg.Plan(shape, dtype=dtype)
    assert mg.mgard_plan_get_tune(plan.handle, 0, 5) >= 0
    t = torch.from_numpy(u).cuda()
    t2 = t.clone()
    plan.decompose(t)
    plan.decompose(t2)
    torch.cuda.synchronize()
    # every element is computed by a fixed thread in a fixed order
    assert torch.equal(t, t2)
    plan.recompose(t)
    torch.cuda.synchronize()
    assert _relerr(t.cpu().numpy().astype(np.float64), u.astype(np.float64)) <= TOL[dtype]


def test_multi_switch():
    mg = _mg()
    plan = mg.Plan((129, 129, 129), dtype="f32")
    assert mg.mgard_plan_get_tune(plan.handle, 0, 4) == 0
    n_coop = plan.launches()
    plan.tune(0, 4, 1)
    assert mg.mgard_plan_get_tune(plan.handle, 0, 4) == 1
    assert mg.mgard_plan_get_tune(plan.handle, 0, 5) == -1
    plan.tune(0, 4, 0)
    assert mg.mgard_plan_get_tune(plan.handle, 0, 5) == 0
    assert plan.launches() == n_coop
    plan.tune(0, 3, 1)  # all tiled wins over the cooperative kernel
    assert mg.mgard_plan_get_tune(plan.handle, 0, 5) == -1
    plan.tune(0, 3, 0)
    assert mg.mgard_plan_get_tune(plan.handle, 0, 5) == 0
    with pytest.raises(mg.MgardError):
        plan.tune(0, 4, 2)


def test_multi_barrier_wait_limit_is_reported():
    """A poll limit far too small for the work between barriers makes waits
    run out: the kernel finishes (every access stays within the level arrays
    whatever the timing), records it, and mgard_plan_check reports it; the
    default limit gives a clean record and the right result."""
    mg = _mg()
    shape = (129, 129, 129)
    u = _field(shape, "f32", 53)
    plan = mg.Plan(shape, dtype="f32")
    ws = plan.workspace("cuda")
    t = torch.from_numpy(u).cuda()
    plan.tune(0, 6, 1)
    assert mg.mgard_plan_get_tune(plan.handle, 0, 6) == 1
    plan.decompose(t, ws)
    with pytest.raises(mg.MgardError) as info:
        plan.check(ws)
    assert info.value.status == 5  # MGARD_ERR_TIMEOUT
    plan.tune(0, 6, 0)
    t = torch.from_numpy(u).cuda()
    plan.decompose(t, ws)
    plan.check(ws)
    want = oracle.decompose(u.astype(np.float64))
    assert _relerr(t.cpu().numpy().astype(np.float64), want) <= TOL["f32"]
    with pytest.raises(mg.MgardError):
        plan.tune(0, 6, -1)
