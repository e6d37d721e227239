"""Every load-vector tile configuration against the FP64 oracle.

Plans run every level with the tiled per-level kernels (tuning parameter 3)
and force configuration 0-3 on each level that can take it (3, the warp
strips, needs >= 30 coarse columns and one strip of coarse rows).  Shapes
have ragged last tiles and strips (97 = 3 x 32 + 1 nodes: 49 coarse rows;
a last strip shifted back over its neighbour), uniform grids (the strips'
shared-row fast path) and non-uniform ones, 2D and 3D, FP32, FP64 and the
mixed scheme.  Tolerances (max relative error): 1e-12 FP64, 1e-5 FP32 and
mixed.
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
    ((65, 97, 129), "f32", False),
    ((65, 97, 129), "f64", True),
    ((129, 65, 257), "f32_mixed", True),
    ((17, 257, 65), "f32", False),
    ((97, 257), "f32", True),
    ((129, 129, 129), "f64", False),
]


@pytest.mark.parametrize("cfg", [0, 1, 2, 3])
@pytest.mark.parametrize("shape,dtype,nonuniform", CASES)
def test_restriction_config_matches_oracle(shape, dtype, nonuniform, cfg):
    mg = _mg()
    coords = _rand_coords(shape, 61) if nonuniform else None
    npdt = np.float64 if dtype == "f64" else np.float32
    u = synth.sinusoid_field(shape, 8, seed=60, dtype=npdt)
    plan = mg.Plan(shape, coords=coords, dtype=dtype)
    plan.tune(0, 3, 1)  # every level with the tiled kernels
    taken = 0
    for level in range(plan.levels):
        try:
            plan.tune(level, 0, cfg)
            taken += 1
        except mg.MgardError:
            assert cfg == 3  # only the strips have a size limit
    assert mg.mgard_plan_get_tune(plan.handle, 0, 0) == cfg and taken >= 1
    want = oracle.decompose(u.astype(np.float64), coords=coords)
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    assert _relerr(t.cpu().numpy().astype(np.float64), want) <= TOL[dtype]
    back = oracle.recompose(want, coords=coords)
    c = torch.from_numpy(want.astype(npdt)).cuda()
    plan.recompose(c)
    torch.cuda.synchronize()
    assert _relerr(c.cpu().numpy().astype(np.float64), back) <= TOL[dtype]
