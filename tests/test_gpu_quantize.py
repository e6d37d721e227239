"""GPU parity of the quantization of the coefficient classes (mgard_quantize,
mgard_dequantize and the combined calls) against the oracle's quantizer
(oracle/quantize.py): the same decomposed field in, bit-identical int32
codes and de-quantized values out (both sides decide every code in the
field's precision), on 1D-3D shapes, FP32, FP64 and the mixed scheme, and on
the full 513^3 FP32 field; the rebuilt field against the oracle's
recomposition of the same de-quantized values."""
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


def _bins(L, scale, seed):
    rng = np.random.default_rng(seed)
    return list(scale * rng.uniform(0.2, 2.0, L + 1) * np.logspace(0, -2, L + 1))


CASES = [((1025,), "f32"), ((129, 65), "f64"), ((65, 33, 129), "f32"), ((33, 17, 65), "f32_mixed"),
         ((17, 257), "f32"), ((9, 9, 9), "f64"), ((3, 5), "f32")]


@pytest.mark.parametrize("shape,dtype", CASES)
def test_codes_and_dequantized_values_bit_exact(shape, dtype):
    mg = _mg()
    u = synth.sinusoid_field(shape, 12, seed=21).astype(_np(dtype))
    plan = mg.Plan(shape, dtype=dtype)
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    c = t.cpu().numpy()                      # the GPU's decomposed field, the input of both quantizers
    bins = _bins(plan.levels, 1e-3 * float(np.abs(u).max()), 22)
    codes = plan.quantize(t, bins)
    torch.cuda.synchronize()
    want = oracle.quantize(c, bins, plan.levels)
    assert np.array_equal(codes.cpu().numpy(), want)
    d = torch.empty_like(t)
    plan.dequantize(codes, bins, d)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), oracle.dequantize(want, bins, plan.levels, c.dtype))


@pytest.mark.parametrize("shape,dtype", [((65, 33, 129), "f32"), ((129, 65), "f64"), ((33, 17, 65), "f32_mixed")])
def test_combined_calls_rebuild_the_oracle_reconstruction(shape, dtype):
    """decompose_quantize then dequantize_recompose: codes equal the separate
    calls' codes, and the rebuilt field equals (to the parity tolerance) the
    oracle's recomposition of the de-quantized coefficients; with every bin
    at 1e-4 max|u| the rebuilt field stays within a few bins of u."""
    mg = _mg()
    u = synth.sinusoid_field(shape, 12, seed=23).astype(_np(dtype))
    plan = mg.Plan(shape, dtype=dtype)
    scale = float(np.abs(u).max())
    bins = [1e-4 * scale] * (plan.levels + 1)
    t = torch.from_numpy(u).cuda()
    codes = plan.decompose_quantize(t, bins)
    torch.cuda.synchronize()
    assert np.array_equal(codes.cpu().numpy(), oracle.quantize(t.cpu().numpy(), bins, plan.levels))
    back = torch.empty_like(t)
    plan.dequantize_recompose(codes, bins, back)
    torch.cuda.synchronize()
    deq = oracle.dequantize(codes.cpu().numpy(), bins, plan.levels, _np(dtype)).astype(np.float64)
    want = oracle.recompose(deq, nlevels=plan.levels)
    got = back.cpu().numpy().astype(np.float64)
    assert np.abs(got - want).max() / np.abs(want).max() <= TOL[dtype]
    assert np.abs(got - u.astype(np.float64)).max() <= 10 * bins[0]


def test_full_size_513_cubed_codes():
    mg = _mg()
    shape = (513, 513, 513)
    plan = mg.Plan(shape, dtype="f32")
    t = synth.sinusoid_field_torch(shape, 12, 2, "cuda", torch.float32)
    plan.decompose(t)
    bins = _bins(plan.levels, 1e-3 * float(t.abs().max()), 24)
    codes = plan.quantize(t, bins)
    torch.cuda.synchronize()
    assert np.array_equal(codes.cpu().numpy(), oracle.quantize(t.cpu().numpy(), bins, plan.levels))


def test_bad_bins_rejected():
    mg = _mg()
    plan = mg.Plan((33, 33), dtype="f32")
    t = torch.zeros((33, 33), device="cuda")
    for bins in ([1.0] * plan.levels + [0.0], [1.0] * plan.levels + [float("nan")]):
        with pytest.raises(mg.MgardError) as e:
            plan.quantize(t, bins)
        assert e.value.status == 1
