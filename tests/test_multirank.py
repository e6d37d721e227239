"""Host logic of the multi-process (N > 1) benchmark on CPU: two gloo ranks.

Under torchrun every rank refactors its own field (independent partitions,
weak scaling, no collective on the data path); the ranks meet at a barrier
around the timed region, the job's time is the slowest rank's, and the
whole-job value counts every rank's bytes.  These tests run the functions
bench.py uses for that (dist_barrier, dist_max, job_gbs) with the gloo
backend on CPU, and the rule that only rank 0 of the reference arm works
and prints.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.dist_barrier(world)
        local_ms = 10.0 + 5.0 * rank           # rank 1 is the slow one
        ms = bench.dist_max(local_ms, world, "cpu")
        q.put((rank, ms, bench.job_gbs(1.0e9, 4, world, ms)))
        bench.dist_barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, gbs in res:
        assert ms == 15.0
        # two ranks x 4 steps x 1 GB in 15 ms
        assert gbs == pytest.approx(2 * 4 * 1.0e9 / 0.015 / 1e9)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    bench.dist_barrier(1)
    assert bench.dist_max(3.5, 1, "cpu") == 3.5
    assert bench.job_gbs(2.0e9, 5, 1, 10.0) == pytest.approx(1000.0)


def _reference_arm(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--gpus", str(world), "--steps", "1", "--warmup", "0"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_other_ranks_exit_without_work():
    r = _reference_arm(1, 2)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_rank0_prints_one_contract_line():
    r = _reference_arm(0, 1)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["unit"] == "GB/s" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["unit"] == line["unit"]
