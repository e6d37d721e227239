"""GPU parity of the recomposition from the first coefficient classes
(Section I, Fig. 1; Section II-A, overall process) against the FP64 oracle,
element by element on seeded inputs, through the C ABI.

The input is the oracle's decomposition of a seeded field, rounded to the
plan's storage type; both sides rebuild from the same rounded classes.
Tolerance as for the full recomposition (max relative error over the whole
array): 1e-12 for FP64, 1e-5 for FP32 and the mixed scheme.
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
        h = rng.uniform(0.5, 1.0, n - 1)
        x = np.concatenate([[0.0], np.cumsum(h)])
        out.append(x / x[-1])
    return out


def _relerr(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


def _classes(plan, coeffs, nclasses, dtype):
    t = torch.from_numpy(np.ascontiguousarray(coeffs)).cuda()
    plan.recompose_classes(t, nclasses)
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


CASES = [
    # shape, dtype, nlevels, nonuniform
    ((129, 129), "f64", -1, False),
    ((1025,), "f32", -1, False),
    ((257,), "f64", 3, True),
    ((65, 33), "f32", -1, True),
    ((33, 33, 33), "f32", -1, False),
    ((65, 65, 65), "f32", -1, False),
    ((33, 65, 97), "f64", -1, False),    # 97 = 3*32+1: ragged rows
    ((17, 65, 33), "f64", 2, True),      # partial level count
    ((65, 129, 65), "f32_mixed", -1, False),
    ((33, 17, 65), "f32_mixed", -1, True),
    ((3, 3, 3), "f32", -1, False),
    ((3,), "f64", -1, False),
]


@pytest.mark.parametrize("shape,dtype,nlevels,nonuniform", CASES)
def test_every_class_count_matches_oracle(shape, dtype, nlevels, nonuniform):
    mg = _mg()
    coords = _rand_coords(shape, 9) if nonuniform else None
    u = synth.sinusoid_field(shape, 8 if len(shape) < 3 else 12, seed=6)
    plan = mg.Plan(shape, nlevels=nlevels, coords=coords, dtype=dtype)
    L = plan.levels
    coeffs = oracle.decompose(u, nlevels=L, coords=coords).astype(_np_dtype(dtype))
    for nc in range(1, L + 2):
        got = _classes(plan, coeffs, nc, dtype)
        want = oracle.recompose_classes(coeffs.astype(np.float64), nc, nlevels=L, coords=coords)
        assert _relerr(got, want) <= TOL[dtype], (nc, _relerr(got, want))


@pytest.mark.parametrize("mode", ["default", "tiled", "single_block"])
@pytest.mark.parametrize("shape,dtype", [((257, 129, 65), "f32"), ((129, 257, 33), "f64")])
def test_level_paths_match_oracle(shape, dtype, mode):
    """Shapes whose coarse end runs in the cooperative kernel: the first
    dropped-level counts start the partial recomposition inside it, later
    ones in the tiled or single-block kernels; the tuning switches force
    the other paths."""
    mg = _mg()
    u = synth.sinusoid_field(shape, 12, seed=7)
    plan = mg.Plan(shape, dtype=dtype)
    if mode == "tiled":
        plan.tune(0, 3, 1)
    elif mode == "single_block":
        plan.tune(0, 4, 1)
    L = plan.levels
    coeffs = oracle.decompose(u, nlevels=L).astype(_np_dtype(dtype))
    for nc in (1, 2, L - 2, L - 1, L, L + 1):
        got = _classes(plan, coeffs, nc, dtype)
        want = oracle.recompose_classes(coeffs.astype(np.float64), nc, nlevels=L)
        assert _relerr(got, want) <= TOL[dtype], (nc, _relerr(got, want))
    plan.check()


def test_all_classes_is_the_recomposition_bitwise():
    mg = _mg()
    shape = (65, 65, 65)
    u = synth.sinusoid_field(shape, 12, seed=8).astype(np.float32)
    plan = mg.Plan(shape, dtype="f32")
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    a = t.clone()
    plan.recompose(t)
    plan.recompose_classes(a, plan.levels + 1)
    torch.cuda.synchronize()
    assert torch.equal(a, t)


def test_dropped_classes_do_not_enter_the_result():
    """Overwriting the coefficients of the omitted classes with anything
    gives the same bits."""
    mg = _mg()
    shape = (33, 65, 33)
    u = synth.sinusoid_field(shape, 12, seed=9).astype(np.float32)
    plan = mg.Plan(shape, dtype="f32")
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    for nc in (1, 3, plan.levels):
        s = 1 << (plan.levels + 1 - nc)
        a, b = t.clone(), t.clone()
        keep = torch.zeros(shape, dtype=torch.bool, device="cuda")
        keep[::s, ::s, ::s] = True
        b[~keep] = 1.0e6
        plan.recompose_classes(a, nc)
        plan.recompose_classes(b, nc)
        torch.cuda.synchronize()
        assert torch.equal(a, b), nc


def test_class_count_range():
    mg = _mg()
    plan = mg.Plan((17, 17), dtype="f32")
    t = torch.zeros((17, 17), device="cuda")
    for bad in (0, plan.levels + 2):
        with pytest.raises(mg.MgardError) as e:
            plan.recompose_classes(t, bad)
        assert e.value.status == 1


def test_full_size_513_cubed_fp32_finest_class_dropped():
    """513^3 FP32 in the benchmark's plan: the finest class and the two
    finest classes left out, against the FP64 oracle on the same classes."""
    mg = _mg()
    shape = (513, 513, 513)
    u = synth.sinusoid_field(shape, 12, seed=2, dtype=np.float32)
    plan = mg.Plan(shape, dtype="f32")
    L = plan.levels
    coeffs = oracle.decompose(u.astype(np.float64)).astype(np.float32)
    for nc in (L, L - 1):
        got = _classes(plan, coeffs, nc, "f32")
        want = oracle.recompose_classes(coeffs.astype(np.float64), nc)
        assert _relerr(got, want) <= 1e-5, (nc, _relerr(got, want))
