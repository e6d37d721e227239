"""The persistent batch kernel's host scheduler (csrc/persist_sched.h), on
the CPU: tests/host/persist_sched_check.cpp builds the tasks of synthetic
fields (a cube with a small tail, uneven sides, a two-dimensional field run
by rows, per-dimension level counts), schedules them on 1, 7 and 304
workers in both queue orders and both directions, and checks that every
item is queued once and after all items it depends on, that item counts per
kind follow the level geometry, that one worker's makespan is the sum of all
item costs and more workers never take longer, and that a reordered queue is
rejected."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_persistent_scheduler_invariants(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = tmp_path / "persist_sched_check"
    cmd = [gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2007_04457_gb300", "csrc"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
           os.path.join(ROOT, "tests", "host", "persist_sched_check.cpp"), "-o", str(exe)]
    subprocess.run(cmd, check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = out.stdout.strip().splitlines()
    assert lines[-1] == "ALL OK"
    assert sum(l.startswith("ok ") for l in lines) >= 40
