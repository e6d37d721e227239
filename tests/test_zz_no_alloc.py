"""mgard_decompose_noalloc (tables and workspace in the library's static
scratch) against the plan-based mgard_decompose, through the C ABI.

Two calls in a row on fresh copies of the field must each match the regular
entry point within the parity tolerance (max relative error over the array:
1e-5 FP32 / mixed, 1e-12 FP64); a shape beyond the scratch is rejected with
MGARD_ERR_WORKSPACE and leaves the field untouched; a call on a stream under
capture is refused with MGARD_ERR_INVALID_ARG.  This file is collected last
so that it also runs after every other GPU test in the same process.
"""
import numpy as np
import pytest

import oracle
from paper_2007_04457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f32_mixed": 1e-5}
INVALID_ARG = 1
WORKSPACE = 3


def _mg():
    from paper_2007_04457_gb300 import mgard
    return mgard


def _relerr(got, want):
    got = got.double()
    want = want.double()
    return float((got - want).abs().max() / want.abs().max().clamp_min(1e-300))


def _noalloc(mg, t, nlevels, dtype):
    mg.mgard_decompose_noalloc(t.dim(), t.shape, nlevels, mg._DTYPE_CODES[dtype], t.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)


CASES = [
    ((257, 257, 257), "f32", -1),
    ((33, 65, 33), "f32", -1),
    ((129, 129), "f64", -1),
    ((257, 129), "f32_mixed", -1),
    ((1025,), "f32", -1),
    ((17, 33, 17), "f64", 2),
]


@pytest.mark.parametrize("shape,dtype,nlevels", CASES)
def test_noalloc_matches_decompose_twice(shape, dtype, nlevels):
    mg = _mg()
    npdt = np.float64 if dtype == "f64" else np.float32
    u = torch.from_numpy(synth.sinusoid_field(shape, 12, seed=7, dtype=npdt)).cuda()
    plan = mg.Plan(shape, nlevels=nlevels, dtype=dtype)
    want = plan.decompose(u.clone())
    for _ in range(2):
        got = u.clone()
        _noalloc(mg, got, nlevels, dtype)
        torch.cuda.synchronize()
        assert _relerr(got, want) <= TOL[dtype]


def test_noalloc_matches_oracle_small():
    mg = _mg()
    shape = (33, 17, 65)
    u = synth.sinusoid_field(shape, 12, seed=8, dtype=np.float32)
    t = torch.from_numpy(u).cuda()
    _noalloc(mg, t, -1, "f32")
    want = oracle.decompose(u.astype(np.float64))
    got = t.cpu().numpy().astype(np.float64)
    assert np.abs(got - want).max() / np.abs(want).max() <= 1e-5


def test_noalloc_rejects_shape_beyond_scratch():
    mg = _mg()
    shape = (4097, 4097)  # FP32 workspace about 45 MB > 32 MiB
    t = torch.full(shape, 1.5, device="cuda")
    with pytest.raises(mg.MgardError) as e:
        _noalloc(mg, t, -1, "f32")
    assert e.value.status == WORKSPACE
    assert "static scratch" in str(e.value)
    torch.cuda.synchronize()
    assert bool((t == 1.5).all())
    # the scratch is still usable afterwards
    small = torch.from_numpy(synth.sinusoid_field((65, 65), 12, seed=9, dtype=np.float32)).cuda()
    want = mg.Plan((65, 65), dtype="f32").decompose(small.clone())
    _noalloc(mg, small, -1, "f32")
    torch.cuda.synchronize()
    assert _relerr(small, want) <= TOL["f32"]


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")  # nothing is queued: the refusal is the point
def test_noalloc_refuses_stream_capture():
    """The call uploads its tables from host memory it frees on return, so it
    refuses a stream under capture before queueing anything; afterwards it
    works as before."""
    mg = _mg()
    shape = (33, 33, 33)
    u = torch.from_numpy(synth.sinusoid_field(shape, 12, seed=10, dtype=np.float32)).cuda()
    t = u.clone()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.graph(g, stream=s):
        try:
            mg.mgard_decompose_noalloc(t.dim(), t.shape, -1, mg._DTYPE_CODES["f32"], t.data_ptr(), s.cuda_stream)
        except mg.MgardError as e:
            status = e.status
    assert status == INVALID_ARG
    torch.cuda.synchronize()
    assert bool((t == u).all())
    want = mg.Plan(shape, dtype="f32").decompose(u.clone())
    _noalloc(mg, t, -1, "f32")
    torch.cuda.synchronize()
    assert _relerr(t, want) <= TOL["f32"]
