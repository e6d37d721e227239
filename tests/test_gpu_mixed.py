"""Mixed precision (FP32 field, FP64 solves and coarse-level arrays) against
the FP64 oracle, with the error reported per level.

Per-level error: for the coefficients of level l (the nodes of
N_l \\ N_{l-1}) and for the coarsest values, max|gpu - oracle| / max|u| and
the RMS of (gpu - oracle) / max|u|.  The mixed scheme keeps every coarse
array and correction in FP64, so its coarse levels are closer to the oracle
than the plain FP32 path's; both stay within the 1e-5 bound.
"""
import numpy as np
import pytest

import oracle
from paper_2007_04457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def level_masks(shape, L):
    """Boolean masks of N_l \\ N_{l-1} for l = L..1, and of N_0."""
    out = {}
    for l in range(L, -1, -1):
        s = 1 << (L - l)
        on = np.ones(shape, dtype=bool)
        coarse = np.ones(shape, dtype=bool)
        for k, n in enumerate(shape):
            idx = np.arange(n)
            sh = [1] * len(shape)
            sh[k] = n
            on &= (idx % s == 0).reshape(sh)
            coarse &= (idx % (2 * s) == 0).reshape(sh)
        out[l] = on & ~coarse if l > 0 else on
    return out


def per_level_errors(got, want, L, scale):
    rows = {}
    for l, m in level_masks(got.shape, L).items():
        d = (got[m] - want[m]) / scale
        rows[l] = (float(np.abs(d).max()), float(np.sqrt(np.mean(d * d))))
    return rows


def test_mixed_precision_per_level_errors():
    from paper_2007_04457_gb300 import mgard
    shape = (257, 257, 129)
    u = synth.sinusoid_field(shape, 12, seed=3, blob=True, dtype=np.float32)
    want = oracle.decompose(u.astype(np.float64))
    scale = float(np.abs(u).max())
    errs = {}
    for dtype in ("f32", "f32_mixed"):
        plan = mgard.Plan(shape, dtype=dtype)
        t = torch.from_numpy(u).cuda()
        plan.decompose(t)
        torch.cuda.synchronize()
        errs[dtype] = per_level_errors(t.cpu().numpy().astype(np.float64), want, plan.levels, scale)
        L = plan.levels
    print("\nlevel  f32 max / rms            mixed max / rms")
    for l in range(L, -1, -1):
        a, b = errs["f32"][l], errs["f32_mixed"][l]
        print(f"{l:5d}  {a[0]:.2e} / {a[1]:.2e}    {b[0]:.2e} / {b[1]:.2e}")
    for dtype in errs:
        assert max(v[0] for v in errs[dtype].values()) <= 1e-5
    # the FP64 coarse arrays pay off on the coarse levels
    coarse = lambda e: sum(e[l][1] ** 2 for l in range(0, 3))
    assert coarse(errs["f32_mixed"]) <= coarse(errs["f32"])


def test_mixed_precision_sides_1025_against_oracle():
    """1025 x 1025 x 65: two sides of 1025 nodes, where the mixed scheme's
    FP64 coarse arrays and solves matter most (6 levels), against the FP64
    oracle: every level within 1e-5 of max|u|, and the recomposition of the
    oracle's coefficients back to the field."""
    from paper_2007_04457_gb300 import mgard
    shape = (1025, 1025, 65)
    u = synth.sinusoid_field(shape, 12, seed=3, blob=True, dtype=np.float32)
    want = oracle.decompose(u.astype(np.float64))
    scale = float(np.abs(u).max())
    plan = mgard.Plan(shape, dtype="f32_mixed")
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    errs = per_level_errors(t.cpu().numpy().astype(np.float64), want, plan.levels, scale)
    print("\nlevel  mixed max / rms (1025 x 1025 x 65)")
    for l in range(plan.levels, -1, -1):
        print(f"{l:5d}  {errs[l][0]:.2e} / {errs[l][1]:.2e}")
    assert max(v[0] for v in errs.values()) <= 1e-5
    t.copy_(torch.from_numpy(want.astype(np.float32)))
    plan.recompose(t)
    torch.cuda.synchronize()
    back = t.cpu().numpy().astype(np.float64)
    assert np.abs(back - u).max() / scale <= 1e-5
