"""Batched fields as a CUDA graph of per-field launches (tuning param 0 =
0) and the autotuner, on the GPU.  The persistent form is covered by
test_gpu_persist.py."""
import numpy as np
import pytest

import oracle
from paper_2007_04457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mg():
    from paper_2007_04457_gb300 import mgard
    return mgard


SHAPES = [(17, 17, 17), (33, 33, 33), (65, 65, 65), (17, 33, 65), (129, 129), (257,), (33, 33, 33)]


def test_batch_equals_single_fields_and_oracle(tmp_path):
    mg = _mg()
    plans = [mg.Plan(s, dtype="f32") for s in SHAPES]
    host = [synth.sinusoid_field(s, 12 if len(s) == 3 else 8, seed=40 + i, dtype=np.float32)
            for i, s in enumerate(SHAPES)]
    fields = [torch.from_numpy(h).cuda() for h in host]
    single = [f.clone() for f in fields]
    batch = mg.Batch(plans, streams=4)
    batch.tune(0, 0)
    assert batch.get("persistent") == 0
    for _ in range(2):  # the second call replays the captured graph
        work = [f.clone() for f in fields]
        batch.decompose(work)
        torch.cuda.synchronize()
    # a batch runs every field with the per-field kernels (no cooperative
    # launch); the same plans with the cooperative kernel switched off give
    # the same bits
    for p, s in zip(plans, single):
        p.tune(0, 4, 1)
        p.decompose(s)
    torch.cuda.synchronize()
    for w, s, h in zip(work, single, host):
        assert torch.equal(w, s)
        want = oracle.decompose(h.astype(np.float64))
        got = w.cpu().numpy().astype(np.float64)
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    batch.recompose(work)
    torch.cuda.synchronize()
    for w, h in zip(work, host):
        assert np.abs(w.cpu().numpy() - h).max() <= 1e-5 * np.abs(h).max()


def test_batch_recaptures_for_new_pointers():
    mg = _mg()
    plans = [mg.Plan(s, dtype="f32") for s in SHAPES[:3]]
    batch = mg.Batch(plans, streams=2)
    batch.tune(0, 0)
    a = [torch.randn(p.shape, device="cuda") for p in plans]
    b = [x.clone() for x in a]
    batch.decompose(a)
    batch.decompose(b)  # other pointers: a new graph
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_autotune_keeps_results(tmp_path):
    from paper_2007_04457_gb300 import autotune
    mg = _mg()
    shape = (65, 129, 65)
    plan = mg.Plan(shape, dtype="f32")
    best = autotune.tune(plan, top=2, reps=1, cache_path=str(tmp_path / "t.json"))
    assert best["cfg"] in (autotune.DEFAULT,) + autotune.CONFIGS and best["warps"] in autotune.SOLVE_WARPS
    u = synth.sinusoid_field(shape, 12, seed=41, dtype=np.float32)
    t = torch.from_numpy(u).cuda()
    plan.decompose(t)
    torch.cuda.synchronize()
    want = oracle.decompose(u.astype(np.float64))
    assert np.abs(t.cpu().numpy() - want).max() <= 1e-5 * np.abs(want).max()
    again = autotune.tune(plan, cache_path=str(tmp_path / "t.json"))
    assert again["cached"] and again["cfg"] == best["cfg"]
