"""The persistent batch kernel: every level of every field of a batch in one
launch per direction, its blocks pulling work items from a device queue.

Parity with the FP64 oracle per field (FP32 1e-5, FP64 1e-12, the mixed
scheme 1e-5) on batches that mix 3D and 2D fields, uneven sizes, graded
coordinates, partial level counts, fields with and without a small tail and
a 1D field; agreement with the graph of per-field launches; a grid of one
block per SM; new pointers (a new level table); a wait that runs out on
purpose (test hook) and is reported as MGARD_ERR_TIMEOUT; a batch the
persistent kernel cannot take; and a sample of the seeded 256-field batch.
"""
import numpy as np
import pytest

import oracle
from paper_2007_04457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-12, "f32_mixed": 1e-5}
TIMEOUT = 5


def _mg():
    from paper_2007_04457_gb300 import mgard
    return mgard


def _np(dtype):
    return np.float64 if dtype == "f64" else np.float32


def _coords(shape, seed):
    rng = np.random.default_rng(seed)
    out = []
    for n in shape:
        h = rng.uniform(0.5, 1.0, n - 1)
        x = np.concatenate([[0.0], np.cumsum(h)])
        out.append(x / x[-1])
    return out


def _relerr(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


# shape, levels (-1 = all), graded coordinates
MIX = [
    ((17, 17, 17), -1, False),
    ((33, 65, 17), -1, False),     # uneven sides: planes of 65 x 17
    ((65, 65, 65), 3, True),       # partial level count, graded grid: no small tail
    ((129, 129), -1, False),       # 2D: rows as planes
    ((257, 65), -1, True),
    ((9, 9, 9), -1, False),        # one grid level, then the small tail
    ((513,), -1, False),           # 1D
    ((129, 33, 257), 2, False),    # rows of 257 nodes
]


def _make(mg, dtype, cases, seed=3):
    plans, host, coords = [], [], []
    for i, (shape, nl, graded) in enumerate(cases):
        c = _coords(shape, seed + i) if graded else None
        plans.append(mg.Plan(shape, nlevels=nl, coords=c, dtype=dtype))
        host.append(synth.sinusoid_field(shape, 12 if len(shape) == 3 else 8, seed=seed + i).astype(_np(dtype)))
        coords.append(c)
    return plans, host, coords


def _dev(host):
    return [torch.from_numpy(np.ascontiguousarray(h)).cuda() for h in host]


@pytest.mark.parametrize("dtype", ["f32", "f64", "f32_mixed"])
def test_persistent_batch_matches_oracle(dtype):
    mg = _mg()
    plans, host, coords = _make(mg, dtype, MIX)
    batch = mg.Batch(plans)
    assert batch.get("eligible") == 1 and batch.get("persistent") == 1
    fields = _dev(host)
    batch.decompose(fields)
    torch.cuda.synchronize()
    assert batch.check() == 0
    coef = []
    for f, h, p, c in zip(fields, host, plans, coords):
        want = oracle.decompose(h.astype(np.float64), nlevels=p.levels, coords=c)
        got = f.cpu().numpy().astype(np.float64)
        assert _relerr(got, want) <= TOL[dtype], (p.shape, _relerr(got, want))
        coef.append(want)
    # recomposition of the oracle's coefficients
    work = _dev([w.astype(_np(dtype)) for w in coef])
    batch.recompose(work)
    torch.cuda.synchronize()
    assert batch.check() == 0
    for f, w, p, c in zip(work, coef, plans, coords):
        want = oracle.recompose(w.astype(_np(dtype)).astype(np.float64), nlevels=p.levels, coords=c)
        got = f.cpu().numpy().astype(np.float64)
        assert _relerr(got, want) <= TOL[dtype], (p.shape, _relerr(got, want))


def test_persistent_agrees_with_per_field_graph_and_repeats():
    mg = _mg()
    plans, host, _ = _make(mg, "f32", MIX, seed=11)
    batch = mg.Batch(plans, streams=4)
    a = _dev(host)
    b = _dev(host)
    batch.decompose(a)
    batch.decompose(b)  # replay: counters reset by the graph
    batch.tune(0, 0)
    g = _dev(host)
    batch.decompose(g)
    torch.cuda.synchronize()
    for x, y, z in zip(a, b, g):
        assert torch.equal(x, y)
        assert _relerr(x.cpu().numpy().astype(np.float64), z.cpu().numpy().astype(np.float64)) <= 2e-5
    batch.tune(0, 1)
    batch.recompose(a)
    torch.cuda.synchronize()
    for x, h in zip(a, host):
        assert _relerr(x.cpu().numpy().astype(np.float64), h.astype(np.float64)) <= 2e-5


def test_one_block_per_sm_and_new_pointers():
    mg = _mg()
    plans, host, coords = _make(mg, "f32", MIX[:5], seed=21)
    batch = mg.Batch(plans)
    batch.tune(3, 1)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert batch.get("grid") == sms and batch.get("blocks_per_sm_req") == 1
    for _ in range(2):  # two sets of pointers: two level tables
        fields = _dev(host)
        batch.decompose(fields)
        torch.cuda.synchronize()
        for f, h, p, c in zip(fields, host, plans, coords):
            want = oracle.decompose(h.astype(np.float64), nlevels=p.levels, coords=c)
            assert _relerr(f.cpu().numpy().astype(np.float64), want) <= 1e-5
    assert batch.check() == 0


def test_wait_that_runs_out_reports_timeout():
    """The test hook makes the first item wait for a count that nothing
    reaches; with a short poll limit the wait gives up, the block goes on,
    and the check reports MGARD_ERR_TIMEOUT.  Without the hook the same
    batch is exact again and the check is clean."""
    mg = _mg()
    plans, host, coords = _make(mg, "f32", MIX[:3], seed=31)
    batch = mg.Batch(plans)
    spin = batch.get("spin")
    batch.tune(1, 2000)
    batch.tune(2, 1)
    fields = _dev(host)
    batch.decompose(fields)
    torch.cuda.synchronize()
    assert batch.check() == TIMEOUT
    assert batch.check() == 0  # the record is cleared
    batch.tune(2, 0)
    batch.tune(1, spin)
    fields = _dev(host)
    batch.decompose(fields)
    torch.cuda.synchronize()
    assert batch.check() == 0
    for f, h, p, c in zip(fields, host, plans, coords):
        want = oracle.decompose(h.astype(np.float64), nlevels=p.levels, coords=c)
        assert _relerr(f.cpu().numpy().astype(np.float64), want) <= 1e-5


def test_batch_the_persistent_kernel_cannot_take():
    mg = _mg()
    plans = [mg.Plan((17, 2049), dtype="f32"), mg.Plan((17, 17, 17), dtype="f32")]
    batch = mg.Batch(plans)
    assert batch.get("eligible") == 0 and batch.get("persistent") == 0
    with pytest.raises(mg.MgardError):
        batch.tune(0, 1)
    host = [synth.sinusoid_field(p.shape, 8, seed=50 + i, dtype=np.float32) for i, p in enumerate(plans)]
    fields = _dev(host)
    batch.decompose(fields)
    torch.cuda.synchronize()
    for f, h, p in zip(fields, host, plans):
        want = oracle.decompose(h.astype(np.float64), nlevels=p.levels)
        assert _relerr(f.cpu().numpy().astype(np.float64), want) <= 1e-5


def test_seeded_uneven_batch_sample_matches_oracle():
    """The 256 fields of uneven dyadic sizes (240 cubes with sides from
    {17, 33, 65, 129, 257}, 16 fields of 1025 x 1025) in one launch per
    direction; the oracle checks one field of every size."""
    mg = _mg()
    shapes = synth.batch_shapes(seed=4)
    plans = [mg.Plan(s, dtype="f32") for s in shapes]
    batch = mg.Batch(plans)
    assert batch.get("persistent") == 1
    fields = [synth.sinusoid_field_torch(s, 12 if len(s) == 3 else 8, 4 + i, "cuda", torch.float32)
              for i, s in enumerate(shapes)]
    pick = {}
    for i, s in enumerate(shapes):
        pick.setdefault(s, i)
    keep = {i: fields[i].cpu().numpy() for i in pick.values()}
    ws = batch.workspace("cuda")
    batch.decompose(fields, ws)
    torch.cuda.synchronize()
    assert batch.check() == 0
    for i, u in keep.items():
        want = oracle.decompose(u.astype(np.float64), nlevels=plans[i].levels)
        got = fields[i].cpu().numpy().astype(np.float64)
        assert _relerr(got, want) <= 1e-5, (shapes[i], _relerr(got, want))
    batch.recompose(fields, ws)
    torch.cuda.synchronize()
    assert batch.check() == 0
    for i, u in keep.items():
        assert _relerr(fields[i].cpu().numpy().astype(np.float64), u.astype(np.float64)) <= 1e-5
