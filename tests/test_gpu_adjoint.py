"""GPU adjoints: the transposed maps against the FP64 oracle's transposes,
dot-product tests, and the autograd gradient of the masked reconstruction
loss against finite differences and the oracle.

Tolerances (max relative error over the array): 1e-12 FP64, 1e-5 FP32 /
mixed for the transposed maps themselves.  The loss gradient
2 (D^T (mask * R^T r) - r), r = R(mask * D u) - u, is a small residual
(|r| ~ 1e-3 |u| for this input) formed from O(|u|) FP32 quantities, so its
FP32 relative error is about eps_32 |u| / |r| ~ 1e-4; the test allows 1e-3.
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


CASES = [
    ((129, 129), "f64", -1, False),
    ((129, 65, 65), "f32", -1, True),   # tiled finest level, then one block
    ((65,), "f32", -1, True),
    ((33, 65), "f32", -1, False),
    ((17, 33, 17), "f64", -1, True),
    ((33, 33, 33), "f32", -1, False),
    ((33, 17, 65), "f32_mixed", -1, False),
    ((17, 17, 33), "f64", 2, False),
    ((3, 3, 3), "f32", -1, False),
]


@pytest.mark.parametrize("shape,dtype,nlevels,nonuniform", CASES)
@pytest.mark.parametrize("which", ["decompose", "recompose"])
@pytest.mark.parametrize("tiled", [False, True])
def test_adjoint_matches_oracle(shape, dtype, nlevels, nonuniform, which, tiled):
    """tiled: every level with the per-level adjoint kernels (tuning parameter
    3); else the levels that fit one block's shared memory run in one launch."""
    mg = _mg()
    coords = _rand_coords(shape, 21) if nonuniform else None
    y = np.random.default_rng(22).standard_normal(shape).astype(_np_dtype(dtype))
    plan = mg.Plan(shape, nlevels=nlevels, coords=coords, dtype=dtype)
    if tiled:
        plan.tune(0, 3, 1)
    t = torch.from_numpy(y).cuda()
    getattr(plan, f"{which}_adjoint")(t)
    torch.cuda.synchronize()
    got = t.cpu().numpy().astype(np.float64)
    want = getattr(oracle, f"{which}_adjoint")(y.astype(np.float64), nlevels=plan.levels, coords=coords)
    assert _relerr(got, want) <= TOL[dtype], _relerr(got, want)


@pytest.mark.parametrize("shape", [(33, 17, 65), (129, 65)])
def test_dot_products_on_gpu(shape):
    """<D x, y> = <x, D^T y> and <R x, y> = <x, R^T y> in FP64."""
    mg = _mg()
    rng = np.random.default_rng(23)
    plan = mg.Plan(shape, dtype="f64")
    x = torch.from_numpy(rng.standard_normal(shape)).cuda()
    y = torch.from_numpy(rng.standard_normal(shape)).cuda()
    for fwd, adj in (("decompose", "decompose_adjoint"), ("recompose", "recompose_adjoint")):
        dx = getattr(plan, fwd)(x.clone())
        dty = getattr(plan, adj)(y.clone())
        lhs = float((dx * y).sum())
        rhs = float((x * dty).sum())
        assert abs(lhs - rhs) <= 1e-12 * float(dx.norm()) * float(y.norm())


def _loss_oracle_grad(u64, mask):
    d = oracle.decompose(u64)
    r = oracle.recompose(mask * d) - u64
    g = oracle.decompose_adjoint(mask * oracle.recompose_adjoint(r)) - r
    return float((r * r).sum()), 2.0 * g


def test_loss_gradient_finite_differences_fp64():
    """Central differences with eps = 1e-3 along a random direction; the loss
    is quadratic, so they are exact up to rounding."""
    from paper_2007_04457_gb300 import autograd as ag
    mg = _mg()
    shape = (17, 33, 17)
    plan = mg.Plan(shape, dtype="f64")
    u = torch.from_numpy(synth.sinusoid_field(shape, 12, seed=5)).cuda().requires_grad_(True)
    mask = torch.from_numpy(synth.keep_mask(shape, seed=5).astype(np.float64)).cuda()
    loss = ag.masked_reconstruction_loss(u, plan, mask)
    loss.backward()
    d = torch.from_numpy(np.random.default_rng(24).standard_normal(shape)).cuda()
    eps = 1e-3
    with torch.no_grad():
        lp = ag.masked_reconstruction_loss(u + eps * d, plan, mask)
        lm = ag.masked_reconstruction_loss(u - eps * d, plan, mask)
    fd = float((lp - lm) / (2 * eps))
    an = float((u.grad * d).sum())
    assert abs(fd - an) <= 1e-8 * max(abs(an), 1e-300)


def test_loss_gradient_finite_differences_fp32():
    """FP32 field, loss accumulated in FP64, eps = 1e-3."""
    from paper_2007_04457_gb300 import autograd as ag
    mg = _mg()
    shape = (33, 33, 33)
    plan = mg.Plan(shape, dtype="f32")
    u = torch.from_numpy(synth.sinusoid_field(shape, 12, seed=5, dtype=np.float32)).cuda().requires_grad_(True)
    mask = torch.from_numpy(synth.keep_mask(shape, seed=5).astype(np.float32)).cuda()
    loss = ag.masked_reconstruction_loss(u, plan, mask)
    loss.backward()
    d = torch.from_numpy(np.random.default_rng(25).standard_normal(shape).astype(np.float32)).cuda()
    eps = 1e-3

    def lossd(v):
        r = ag.recompose(mask * ag.decompose(v, plan), plan) - v
        return float((r.double() ** 2).sum())

    with torch.no_grad():
        fd = (lossd(u + eps * d) - lossd(u - eps * d)) / (2 * eps)
    an = float((u.grad.double() * d.double()).sum())
    assert abs(fd - an) <= 2e-2 * abs(an)


def test_loss_gradient_257_cubed_fp32_matches_oracle():
    """257^3 FP32, 10% keep-mask on the finest coefficients: autograd through
    the adjoint kernels against the oracle's transposes in FP64."""
    from paper_2007_04457_gb300 import autograd as ag
    mg = _mg()
    shape = (257, 257, 257)
    u32 = synth.sinusoid_field(shape, 12, seed=5, dtype=np.float32)
    m = synth.keep_mask(shape, seed=5)
    plan = mg.Plan(shape, dtype="f32")
    u = torch.from_numpy(u32).cuda().requires_grad_(True)
    mask = torch.from_numpy(m.astype(np.float32)).cuda()
    loss = ag.masked_reconstruction_loss(u, plan, mask)
    loss.backward()
    got = u.grad.cpu().numpy().astype(np.float64)
    lref, want = _loss_oracle_grad(u32.astype(np.float64), m.astype(np.float64))
    assert abs(float(loss.detach()) - lref) <= 1e-3 * lref
    assert _relerr(got, want) <= 1e-3, _relerr(got, want)
