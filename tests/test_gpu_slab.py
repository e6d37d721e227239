"""GPU parity of the slab load-vector kernel (a block per band of coarse rows
x chunk of coarse planes, whole rows staged in shared memory by bulk
asynchronous copies) against the FP64 oracle, and against the strip / tile
kernels it replaces (tuning param 10 = 1 keeps it out).

Every level runs the per-level kernels here (tuning param 3 = 1), so the
slab kernel takes every 3D level with FP32 level arrays and rows of
64 k + 1 nodes, not only the finest.  Shapes cover rows of 129, 257, 513
and 1025 nodes (two to sixteen warps per block), bands of 6 and of 4 coarse
rows (a level with fewer than 6), a last band shifted back over its
neighbour, FP32 and the mixed scheme (FP32 level 0, FP64 coarse arrays),
uniform and graded coordinates and partial level counts, with the solve
along the contiguous dimension left to the solve kernels (the default) and
in the kernel (tuning param 16 = 1, also on every CASES shape); the
chunk, band, ring-slot and register choices are swept on one shape; and a
copy wait that runs out on purpose is reported by mgard_plan_check.
"""
import numpy as np
import pytest

import oracle
from paper_2007_04457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f32_mixed": 1e-5}


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
    # shape, dtype, nlevels, nonuniform
    ((9, 17, 129), "f32", -1, False),         # two warps per block, bands of 6 coarse rows
    ((5, 9, 129), "f32", -1, False),          # 5 coarse rows: bands of 4
    ((17, 33, 257), "f32", -1, True),         # graded grid, levels 0 and 1 by the slab kernel
    ((9, 17, 513), "f32_mixed", -1, False),   # FP64 coarse arrays
    ((33, 65, 129), "f32", 2, False),         # partial level count
    ((5, 17, 1025), "f32", -1, True),         # 256 threads per block
    ((9, 41, 257), "f32", 3, False),          # 21 coarse rows: the last band shifted back
]


def _run(shape, dtype, nlevels, nonuniform, slab_on=True, tune=()):
    mg = _mg()
    coords = _rand_coords(shape, 5) if nonuniform else None
    plan = mg.Plan(shape, nlevels=nlevels, coords=coords, dtype=dtype)
    plan.tune(0, 3, 1)  # per-level kernels on every level
    if not slab_on:
        plan.tune(0, 10, 1)
    for param, value in tune:
        plan.tune(0, param, value)
    return mg, plan, coords


@pytest.mark.parametrize("shape,dtype,nlevels,nonuniform", CASES)
def test_slab_matches_oracle(shape, dtype, nlevels, nonuniform):
    mg, plan, coords = _run(shape, dtype, nlevels, nonuniform)
    assert mg.mgard_plan_get_tune(plan.handle, 0, 12) in (4, 6, 8), "the slab kernel takes level 0"
    u = synth.sinusoid_field(shape, 12, seed=3, dtype=np.float32)
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    plan.check()
    want = oracle.decompose(u.astype(np.float64), nlevels=plan.levels, coords=coords)
    assert _relerr(t.cpu().numpy().astype(np.float64), want) <= TOL[dtype]
    plan.recompose(t)
    torch.cuda.synchronize()
    plan.check()
    assert _relerr(t.cpu().numpy().astype(np.float64), u.astype(np.float64)) <= TOL[dtype]
    # recomposition of the oracle's coefficients (the restriction of stored
    # coefficients on its own)
    c = torch.from_numpy(want.astype(np.float32)).cuda()
    plan.recompose(c)
    torch.cuda.synchronize()
    back = oracle.recompose(want.astype(np.float32).astype(np.float64), nlevels=plan.levels, coords=coords)
    assert _relerr(c.cpu().numpy().astype(np.float64), back) <= TOL[dtype]


@pytest.mark.parametrize("shape,dtype,nlevels,nonuniform", CASES)
def test_slab_with_dim2_solve_matches_oracle(shape, dtype, nlevels, nonuniform):
    mg, plan, coords = _run(shape, dtype, nlevels, nonuniform, tune=((16, 1),))
    assert mg.mgard_plan_get_tune(plan.handle, 0, 16) == 1
    u = synth.sinusoid_field(shape, 12, seed=9, dtype=np.float32)
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    want = oracle.decompose(u.astype(np.float64), nlevels=plan.levels, coords=coords)
    assert _relerr(t.cpu().numpy().astype(np.float64), want) <= TOL[dtype]
    plan.recompose(t)
    torch.cuda.synchronize()
    assert _relerr(t.cpu().numpy().astype(np.float64), u.astype(np.float64)) <= TOL[dtype]


@pytest.mark.parametrize("shape,dtype,nlevels,nonuniform", CASES[:4])
def test_slab_agrees_with_strip_kernels(shape, dtype, nlevels, nonuniform):
    u = synth.sinusoid_field(shape, 12, seed=4, dtype=np.float32)
    outs = []
    for on in (True, False):
        mg, plan, _ = _run(shape, dtype, nlevels, nonuniform, slab_on=on)
        assert (mg.mgard_plan_get_tune(plan.handle, 0, 12) > 0) == on
        t = torch.from_numpy(u).cuda()
        plan.decompose(t)
        torch.cuda.synchronize()
        outs.append(t.cpu().numpy().astype(np.float64))
    assert _relerr(outs[0], outs[1]) <= 1e-6


@pytest.mark.parametrize("tune", [
    ((11, 1),), ((11, 2),), ((11, 5),), ((11, 40),),       # coarse planes per chunk
    ((13, 2),), ((13, 3),), ((13, 8),),                   # ring slots
    ((12, 4),), ((12, 4), (11, 3), (13, 5)),              # bands of 4 rows
    ((12, 8),), ((12, 8), (15, 2)), ((15, 3),),           # bands of 8 rows; register variants
    ((16, 1),), ((16, 1), (12, 4)), ((16, 1), (12, 8)),   # the dim-2 solve in the kernel
])
def test_slab_launch_shapes(tune):
    shape = (17, 33, 257)
    mg, plan, coords = _run(shape, "f32", -1, True, tune=tune)
    for param, value in tune:
        if param == 11:
            assert mg.mgard_plan_get_tune(plan.handle, 0, 11) == min(value, (shape[0] - 1) // 2)
        elif param in (12, 13, 15, 16):
            assert mg.mgard_plan_get_tune(plan.handle, 0, param) == value
    u = synth.sinusoid_field(shape, 12, seed=6, dtype=np.float32)
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    plan.check()
    want = oracle.decompose(u.astype(np.float64), coords=coords)
    assert _relerr(t.cpu().numpy().astype(np.float64), want) <= 1e-5


def test_slab_full_size_513_cubed_both_directions():
    """The bench's shape and launch configuration (the coarse end in one
    launch): decomposition against the oracle, recomposition back."""
    mg = _mg()
    shape = (513, 513, 513)
    u = synth.sinusoid_field(shape, 12, seed=7, dtype=np.float32)
    plan = mg.Plan(shape, dtype="f32")
    assert mg.mgard_plan_get_tune(plan.handle, 0, 12) > 0
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    plan.check()
    want = oracle.decompose(u.astype(np.float64), nlevels=plan.levels)
    assert _relerr(t.cpu().numpy().astype(np.float64), want) <= 1e-5
    plan.recompose(t)
    torch.cuda.synchronize()
    plan.check()
    assert _relerr(t.cpu().numpy().astype(np.float64), u.astype(np.float64)) <= 1e-5


def test_slab_copy_wait_that_runs_out_is_reported():
    """Test hook (tuning param 14 = wait limit in microseconds): each block's
    first copy is announced with 16 bytes more than it moves, so its phase
    never completes; the wait gives up after the limit, the block records
    it, waits (bounded) for its other copies and returns.  mgard_plan_check
    reports MGARD_ERR_TIMEOUT once; the next call without the hook is
    exact."""
    shape = (9, 17, 129)
    mg, plan, _ = _run(shape, "f32", -1, False)
    assert mg.mgard_plan_get_tune(plan.handle, 0, 12) > 0
    u = synth.sinusoid_field(shape, 12, seed=8, dtype=np.float32)
    plan.tune(0, 14, 1000)
    assert mg.mgard_plan_get_tune(plan.handle, 0, 14) == 1000
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    with pytest.raises(mg.MgardError) as e:
        plan.check()
    assert e.value.status == 5
    plan.check()  # the word was cleared
    plan.tune(0, 14, 0)
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    plan.check()
    want = oracle.decompose(u.astype(np.float64), nlevels=plan.levels)
    assert _relerr(t.cpu().numpy().astype(np.float64), want) <= 1e-5
