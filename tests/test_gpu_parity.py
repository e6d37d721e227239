"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle,
element by element on seeded inputs.

Tolerance (max relative error, max|gpu - oracle| / max|oracle| over the whole
array): 1e-12 for FP64, 1e-5 for FP32 and the mixed scheme.  FP32 runs feed
the oracle the FP32-rounded input widened to FP64.
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


def _np_dtype(dtype):
    return np.float64 if dtype == "f64" else np.float32


def _rand_coords(shape, seed):
    rng = np.random.default_rng(seed)
    out = []
    for n in shape:
        # mildly graded grid: increasing, spacing ratios within [0.5, 2]
        h = rng.uniform(0.5, 1.0, n - 1)
        x = np.concatenate([[0.0], np.cumsum(h)])
        out.append(x / x[-1])
    return out


def _relerr(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


def _gpu(fn_name, plan, host, dtype):
    t = torch.from_numpy(np.ascontiguousarray(host.astype(_np_dtype(dtype)))).cuda()
    getattr(plan, fn_name)(t)
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


CASES = [
    # shape, dtype, nlevels, nonuniform
    ((129, 129), "f64", -1, False),      # 2D 129x129 FP64, 7 levels
    ((1025,), "f32", -1, False),
    ((257,), "f64", 3, True),
    ((65, 33), "f32", -1, True),
    ((17, 257), "f32", -1, False),
    ((33, 33, 33), "f32", -1, False),
    ((65, 65, 65), "f32", -1, False),
    ((33, 65, 97), "f64", -1, False),    # 97 = 3*32+1: 5 levels, ragged tiles
    ((17, 65, 33), "f64", 2, True),
    ((65, 129, 65), "f32_mixed", -1, False),
    ((33, 17, 65), "f32_mixed", -1, True),
    ((1025, 9), "f32", -1, False),      # long strided lines: shared-memory solve
    ((9, 1025), "f64", -1, True),       # long contiguous lines: shared-memory solve
    ((3, 3, 3), "f32", -1, False),
    ((3, 5), "f64", -1, False),
    ((3,), "f32", -1, False),
    ((9, 9, 9), "f64", 0, False),        # zero levels: identity
]


@pytest.mark.parametrize("shape,dtype,nlevels,nonuniform", CASES)
def test_decompose_matches_oracle(shape, dtype, nlevels, nonuniform):
    mg = _mg()
    coords = _rand_coords(shape, 7) if nonuniform else None
    u = synth.sinusoid_field(shape, 8 if len(shape) < 3 else 12, seed=1).astype(_np_dtype(dtype))
    plan = mg.Plan(shape, nlevels=nlevels, coords=coords, dtype=dtype)
    got = _gpu("decompose", plan, u, dtype)
    want = oracle.decompose(u.astype(np.float64), nlevels=plan.levels, coords=coords)
    assert _relerr(got, want) <= TOL[dtype], _relerr(got, want)


@pytest.mark.parametrize("shape,dtype,nlevels,nonuniform", CASES)
def test_recompose_matches_oracle(shape, dtype, nlevels, nonuniform):
    mg = _mg()
    coords = _rand_coords(shape, 8) if nonuniform else None
    u = synth.sinusoid_field(shape, 8 if len(shape) < 3 else 12, seed=2)
    plan = mg.Plan(shape, nlevels=nlevels, coords=coords, dtype=dtype)
    coeffs = oracle.decompose(u, nlevels=plan.levels, coords=coords).astype(_np_dtype(dtype))
    got = _gpu("recompose", plan, coeffs, dtype)
    want = oracle.recompose(coeffs.astype(np.float64), nlevels=plan.levels, coords=coords)
    assert _relerr(got, want) <= TOL[dtype], _relerr(got, want)


@pytest.mark.parametrize("shape,dtype", [((65, 65, 65), "f32"), ((129, 129), "f64"),
                                         ((1025,), "f32_mixed")])
def test_round_trip_on_gpu(shape, dtype):
    mg = _mg()
    u = synth.sinusoid_field(shape, 12, seed=3).astype(_np_dtype(dtype))
    plan = mg.Plan(shape, dtype=dtype)
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    plan.recompose(t)
    torch.cuda.synchronize()
    assert _relerr(t.cpu().numpy().astype(np.float64), u.astype(np.float64)) <= TOL[dtype]


def test_piecewise_linear_input_gives_zero_fine_coefficients():
    """Trilinear data on N_{L-2}: every coefficient of levels L and L-1 is
    zero to rounding on the GPU too."""
    mg = _mg()
    shape = (33, 65, 33)
    coarse = np.random.default_rng(4).integers(-4, 5, size=(9, 17, 9)).astype(np.float64)
    u = coarse
    for k in range(3):
        for _ in range(2):
            n = u.shape[k]
            xi = np.arange(2 * n - 1) / 2.0
            u = np.apply_along_axis(lambda v: np.interp(xi, np.arange(n), v), k, u)
    assert u.shape == shape
    plan = mg.Plan(shape, dtype="f32")
    got = _gpu("decompose", plan, u, "f32")
    mask = np.ones(shape, dtype=bool)
    mask[::4, ::4, ::4] = False
    assert np.abs(got[mask]).max() <= 1e-5 * np.abs(u).max()


def test_workspace_errors():
    mg = _mg()
    plan = mg.Plan((33, 33, 33), dtype="f32")
    t = torch.zeros((33, 33, 33), device="cuda")
    small = torch.empty(plan.workspace_bytes // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(mg.MgardError) as e:
        plan.decompose(t, workspace=small)
    assert e.value.status == 3
    big = torch.empty(plan.workspace_bytes + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(mg.MgardError) as e:
        plan.decompose(t, workspace=big[8:])
    assert e.value.status == 3


def test_full_size_513_cubed_fp32_matches_oracle():
    """513^3 FP32, 9 levels, in the benchmark's launch configuration, against
    the FP64 oracle on the same (FP32-rounded) input."""
    mg = _mg()
    shape = (513, 513, 513)
    u = synth.sinusoid_field(shape, 12, seed=2, dtype=np.float32)
    plan = mg.Plan(shape, dtype="f32")
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    got = t.cpu().numpy()
    want = oracle.decompose(u.astype(np.float64))
    assert _relerr(got.astype(np.float64), want) <= 1e-5
    plan.recompose(t)
    torch.cuda.synchronize()
    back = t.cpu().numpy().astype(np.float64)
    assert _relerr(back, u.astype(np.float64)) <= 1e-5


def test_full_size_513_cubed_fp64_matches_oracle():
    """513^3 FP64, 9 levels (the benchmark's FP64 line), against the FP64
    oracle on the whole array at 1e-12, and the round trip."""
    mg = _mg()
    shape = (513, 513, 513)
    u = synth.sinusoid_field(shape, 12, seed=2, dtype=np.float64)
    plan = mg.Plan(shape, dtype="f64")
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    got = t.cpu().numpy()
    want = oracle.decompose(u)
    assert _relerr(got, want) <= 1e-12
    plan.recompose(t)
    torch.cuda.synchronize()
    assert _relerr(t.cpu().numpy(), u) <= 1e-12
