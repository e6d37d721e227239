"""Host-side rules of bench.py that need no GPU: which source changes
invalidate a recorded DRAM-traffic figure, and the algorithmic byte counts
of the metric."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.fixture
def csrc_copy(tmp_path, monkeypatch):
    dst = tmp_path / "paper_2007_04457_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_2007_04457_gb300", "csrc"), dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return dst


def _touch(path):
    with open(path, "a") as f:
        f.write("\n// edit\n")


INTERP, COEF, RESTRICT = "interpolation sweep", "coefficient sweep", "restriction"


def test_traffic_key_ignores_other_kernels_device_code(csrc_copy):
    before = {k: bench.kernel_source_hash(k) for k in (INTERP, COEF, RESTRICT, "prolong")}
    whole = bench.kernel_source_hash()
    _touch(csrc_copy / "prolong.cuh")
    assert bench.kernel_source_hash(INTERP) == before[INTERP]
    assert bench.kernel_source_hash(COEF) == before[COEF]
    assert bench.kernel_source_hash(RESTRICT) == before[RESTRICT]
    assert bench.kernel_source_hash("prolong") != before["prolong"]
    assert bench.kernel_source_hash() != whole


def test_traffic_key_follows_own_and_shared_sources(csrc_copy):
    before = {k: bench.kernel_source_hash(k) for k in (INTERP, RESTRICT, "prolong")}
    _touch(csrc_copy / "rowchunk.cuh")
    assert bench.kernel_source_hash(INTERP) != before[INTERP]
    assert bench.kernel_source_hash(RESTRICT) == before[RESTRICT]
    assert bench.kernel_source_hash("prolong") == before["prolong"]
    _touch(csrc_copy / "restrict_strip.cuh")             # the strip kernel is no longer the restriction
    assert bench.kernel_source_hash(RESTRICT) == before[RESTRICT]
    _touch(csrc_copy / "slab.cuh")
    assert bench.kernel_source_hash(RESTRICT) != before[RESTRICT]
    mid = {k: bench.kernel_source_hash(k) for k in (INTERP, "prolong")}
    _touch(csrc_copy / "api.cu")   # host code shared by every kernel
    assert all(bench.kernel_source_hash(k) != mid[k] for k in mid)


def test_recorded_traffic_only_for_known_kernels_and_current_sources(csrc_copy, tmp_path):
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_source_hash(INTERP)
    (prof / "traffic.txt").write_text(f"# comment\n{INTERP}\t{h}\t123\n{COEF}\t0000000000000000\t7\n")
    assert bench.recorded_traffic(INTERP) == 123.0
    assert bench.recorded_traffic(COEF) is None        # taken on other sources
    assert bench.recorded_traffic("solve x/y") is None  # no record kept for it
    _touch(csrc_copy / "rowchunk.cuh")
    assert bench.recorded_traffic(INTERP) is None


def test_kernel_groups_join_both_directions_of_the_restriction():
    """The restriction is one kernel in both directions: its two kinds form
    one group whose bytes are the compulsory bytes of each launch."""
    prof = [("restrict_dec", 0, 0, 2, 0.4), ("restrict_rec", 1, 0, 2, 0.4), ("interp", 5, 0, 2, 0.5)]
    g = bench.kernel_groups(prof, (513, 513, 513), 4, 4)
    assert set(g) == {RESTRICT, INTERP}
    assert g[RESTRICT]["launches"] == 4 and g[RESTRICT]["ms"] == pytest.approx(0.8)
    Mf, Mc = 513 ** 3, 257 ** 3
    assert g[RESTRICT]["bytes"] == 4 * (Mf * 4 + 2 * Mc * 4)
    assert g[INTERP]["bytes"] == 2 * (2 * Mf * 4)            # FP32: V costs as much as the coarse nodes
    assert bench.kernel_bytes(5, (513, 513, 513), 4, 8) == 2 * Mf * 4 + Mc * 4   # mixed: V in FP64


def test_fp64_flops_counts_levels():
    """One 3D level of 9^3: 2 x (13 x 729 + 16 x 125) flops."""
    assert bench.fp64_flops((9, 9, 9), 1) == 2 * (13 * 729 + 16 * 125)
    assert bench.fp64_flops((513, 513, 513), 9) == pytest.approx(4.6e9, rel=0.05)


def test_algorithmic_bytes_513_cubed_fp32():
    """2 M_l S per decomposition level, (3 M_l - M_{l-1}) S per recomposition
    level, summed over the 9 levels of 513^3: 1.2355 + 1.7756 GB."""
    dec, rec = bench.algorithmic_bytes((513, 513, 513), 9, 4)
    assert dec == pytest.approx(1.2355e9, rel=1e-4)
    assert rec == pytest.approx(1.7756e9, rel=1e-4)
    M = bench.level_nodes((513, 513, 513), 9)
    assert M[0] == 513 ** 3 and M[1] == 257 ** 3 and M[-1] == 2 ** 3
