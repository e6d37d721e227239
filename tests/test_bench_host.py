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


def test_traffic_key_ignores_other_kernels_device_code(csrc_copy):
    before = {k: bench.kernel_source_hash(k) for k in ("interp", "coef", "prolong")}
    whole = bench.kernel_source_hash()
    _touch(csrc_copy / "prolong.cuh")
    assert bench.kernel_source_hash("interp") == before["interp"]
    assert bench.kernel_source_hash("coef") == before["coef"]
    assert bench.kernel_source_hash("prolong") != before["prolong"]
    assert bench.kernel_source_hash() != whole


def test_traffic_key_follows_own_and_shared_sources(csrc_copy):
    before = {k: bench.kernel_source_hash(k) for k in ("interp", "prolong")}
    _touch(csrc_copy / "sweep.cuh")
    assert bench.kernel_source_hash("interp") != before["interp"]
    assert bench.kernel_source_hash("prolong") == before["prolong"]
    mid = {k: bench.kernel_source_hash(k) for k in ("interp", "prolong")}
    _touch(csrc_copy / "api.cu")   # host code shared by every kernel
    assert all(bench.kernel_source_hash(k) != mid[k] for k in mid)


def test_recorded_traffic_only_for_known_kernels_and_current_sources(csrc_copy, tmp_path):
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_source_hash("interp")
    (prof / "traffic.txt").write_text(f"# comment\ninterp {h} 123\ncoef 0000000000000000 7\n")
    assert bench.recorded_traffic("interp") == 123.0
    assert bench.recorded_traffic("coef") is None       # taken on other sources
    assert bench.recorded_traffic("solve") is None      # no record kept for it
    _touch(csrc_copy / "sweep.cuh")
    assert bench.recorded_traffic("interp") is None


def test_algorithmic_bytes_513_cubed_fp32():
    """2 M_l S per decomposition level, (3 M_l - M_{l-1}) S per recomposition
    level, summed over the 9 levels of 513^3: 1.2355 + 1.7756 GB."""
    dec, rec = bench.algorithmic_bytes((513, 513, 513), 9, 4)
    assert dec == pytest.approx(1.2355e9, rel=1e-4)
    assert rec == pytest.approx(1.7756e9, rel=1e-4)
    M = bench.level_nodes((513, 513, 513), 9)
    assert M[0] == 513 ** 3 and M[1] == 257 ** 3 and M[-1] == 2 ** 3
