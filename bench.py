#!/usr/bin/env python
"""Throughput of the multilevel decomposition + recomposition on GB300.

Workload: one 513^3 FP32 field (seeded sinusoid sum plus noise, 12 modes), the
full 9-level decomposition followed by the full recomposition.  A step is one
decompose + one recompose of the resident field.  The metric is algorithmic
HBM bytes per second:

  decompose level l:   2 M_l S            (read and write the level's nodes)
  recompose level l:   (3 M_l - M_{l-1}) S (coefficients read twice, coarse
                                            values read, level written)

summed over l = L..1, divided by the time of the step (M_l = nodes of level
l, S = bytes per element).  The field (540 MB) is larger than the 129 MB L2,
so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       python bench.py --case SHAPE DTYPE REPS [NCLASSES] [TUNE]   (profiling case)
Under torchrun each rank refactors its own field (independent partitions,
weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHAPE = (513, 513, 513)
N_MODES = 12
E2E_LANES = 3  # fields in flight in the end-to-end leg (2: 394, 3: 440, 4: 449 GB/s measured)
SEED = 2
KIND_NAMES = {0: "restrict_dec", 1: "restrict_rec", 2: "solve", 3: "solve_fused", 8: "small", 9: "multi",
              4: "coef", 5: "interp", 6: "scatter", 7: "adjoint", 10: "prolong"}


def level_nodes(shape, L):
    """M_l for l = L..0 (index 0 = finest)."""
    out = []
    for j in range(L + 1):
        s = 1 << j
        m = 1
        for n in shape:
            m *= (n - 1) // s + 1
        out.append(m)
    return out


def algorithmic_bytes(shape, L, S):
    M = level_nodes(shape, L)
    dec = sum(2 * M[j] * S for j in range(L))
    rec = sum((3 * M[j] - M[j + 1]) * S for j in range(L))
    return dec, rec


def kernel_bytes(kind, shape, S, SW):
    """Compulsory bytes of one finest-level launch of a kernel kind."""
    M = level_nodes(shape, 1)
    Mf, Mc = M[0], M[1]
    return {
        0: Mf * S + 2 * Mc * SW,                   # read level, write F and V
        1: Mf * S + 2 * Mc * SW,                   # read level, write F and V
        2: 2 * Mc * SW,                            # read + write F
        3: 3 * Mc * SW,                            # read F, read + write V
        4: 2 * Mf * S,                             # read + write the level
        5: 2 * Mf * S + Mc * SW,                   # read coefficients + V, write level
        6: Mc * SW + Mc * S,                       # read V, write the coarse nodes
    }[kind]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Headers that hold nothing but the device code of other kernels: a change
# there cannot alter the code, launch or memory traffic of a kernel defined
# elsewhere.  Keys: the kernel names recorded in profiles/traffic.txt.
_OWN_HEADER = {"coef": "sweep.cuh", "interp": "sweep.cuh", "prolong": "prolong.cuh"}
_DEVICE_ONLY_HEADERS = ("adjoint.cuh", "multi.cuh", "prolong.cuh", "restrict.cuh", "restrict_strip.cuh",
                        "small.cuh", "solve.cuh", "sweep.cuh")


def kernel_source_hash(kernel=None):
    """Hash of the library sources (all of them), or of those that define
    one kernel: every source except the device-code headers of other
    kernels."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2007_04457_gb300", "csrc")
    own = _OWN_HEADER.get(kernel)
    for f in sorted(os.listdir(csrc)):
        if kernel is not None and f in _DEVICE_ONLY_HEADERS and f != own:
            continue
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current sources of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path) or kernel_name not in _OWN_HEADER:
        return None
    cur = kernel_source_hash(kernel_name)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel_name and parts[1] == cur:
            return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_barrier(world):
    """Barrier over the ranks (no-op for one process)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def dist_max(x, world, device):
    """Largest value of x over the ranks: the job's time is its slowest rank's.
    `device` is where the reduction tensor lives (the GPU for NCCL, the CPU
    for gloo)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbs(bytes_per_rank_step, steps, world, ms_max):
    """Whole-job GB/s: every rank moves the same bytes per step on its own
    field (weak scaling), in the time of the slowest rank."""
    return world * bytes_per_rank_step * steps / (ms_max / 1e3) / 1e9


def run_reference(args):
    """The oracle (plain FP64 CPU code) on the host cores, same metric."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2007_04457_gb300 import synth

    n = 129
    shape = (n, n, n)
    L = 7
    u = synth.sinusoid_field(shape, N_MODES, SEED, dtype=np.float32).astype(np.float64)
    dec_b, rec_b = algorithmic_bytes(shape, L, 4)
    for _ in range(args.warmup):
        oracle.recompose(oracle.decompose(u))
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.recompose(oracle.decompose(u))
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = (dec_b + rec_b) * args.steps / total / 1e9
    line = {
        "impl": "reference", "metric": "decompose+recompose GB/s (algorithmic bytes) at 513^3 FP32",
        "value": value, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "513^3 FP32 decompose+recompose, 9 levels",
                   "sample": "129^3 sub-grid of the same generator per step, 7 levels"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "129^3, FP64 oracle, one decompose+recompose per step"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_sample():
    """Oracle on a bounded sample (257^3 sub-grid, FP64, one thread)."""
    import numpy as np

    import oracle
    from paper_2007_04457_gb300 import synth

    n = 257
    shape = (n, n, n)
    u = synth.sinusoid_field(shape, N_MODES, SEED, dtype=np.float32).astype(np.float64)
    dec_b, rec_b = algorithmic_bytes(shape, 8, 4)
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.recompose(oracle.decompose(u))
        reps += 1
        if time.perf_counter() - t0 > 8.0 or reps >= 3:
            break
    dt = time.perf_counter() - t0
    return {"value": (dec_b + rec_b) * reps / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"257^3 sub-grid of the same generator, FP64 oracle, {reps} decompose+recompose"}


def _timed(torch, stream, fn, steps):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_batched(torch, mgard, synth, dev, stream, rank):
    """256 FP32 fields of uneven dyadic sizes (240 cubes with sides drawn from
    {17, 33, 65, 129, 257}, 16 fields of 1025 x 1025) refactored by one
    CUDA-graph launch per direction, tile shapes from the autotuner; compared
    with the same fields refactored one by one."""
    from paper_2007_04457_gb300 import autotune

    shapes = synth.batch_shapes(seed=4)
    plans, fields, tuned = [], [], {}
    for i, shp in enumerate(shapes):
        p = mgard.Plan(shp, dtype="f32")
        f = synth.sinusoid_field_torch(shp, 12 if len(shp) == 3 else 8, 4 + i + 1000 * rank, dev, torch.float32)
        if shp not in tuned:
            tuned[shp] = autotune.tune(p, f.clone(), top=2, reps=2)
        else:
            autotune.apply(p, tuned[shp]["cfg"], tuned[shp]["warps"])
        plans.append(p)
        fields.append(f)
    batch = mgard.Batch(plans, streams=8)
    ws = batch.workspace(dev)
    step = lambda: (batch.decompose(fields, ws, stream), batch.recompose(fields, ws, stream))
    for _ in range(3):
        step()
    ms = _timed(torch, stream, step, 5)
    total = 0
    for p in plans:
        d, r = algorithmic_bytes(p.shape, p.levels, 4)
        total += d + r
    # the same fields one at a time, per distinct shape x multiplicity
    single_ms = 0.0
    for shp, cnt in {s: shapes.count(s) for s in set(shapes)}.items():
        i = shapes.index(shp)
        p, f = plans[i], fields[i]
        w = p.workspace(dev)
        one = lambda: (p.decompose(f, w, stream), p.recompose(f, w, stream))
        one()
        single_ms += cnt * _timed(torch, stream, one, 3)
    return {"value": total / (ms / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": ms, "fields": len(shapes),
            "nodes": int(sum(int(np.prod(s)) for s in shapes)), "graph_launches_per_step": 2,
            "single_field_ms_per_step": single_ms, "speedup_vs_single_fields": single_ms / ms,
            "tuned": {"x".join(map(str, k)): [v["cfg"], v["warps"]] for k, v in tuned.items()}}


def run_adjoint(torch, mgard, synth, dev, stream, rank):
    """257^3 FP32, loss ||recompose(mask * decompose(u)) - u||^2 with a fixed
    10% keep-mask on the finest coefficients: forward + backward through the
    hand-written adjoint kernels (torch.autograd), against twice the plain
    decompose + recompose of the same field."""
    import numpy as np

    from paper_2007_04457_gb300 import autograd as ag

    shape = (257, 257, 257)
    plan = mgard.Plan(shape, dtype="f32")
    u0 = synth.sinusoid_field_torch(shape, 12, 5 + rank, dev, torch.float32)
    mask = torch.from_numpy(synth.keep_mask(shape, seed=5).astype(np.float32)).to(dev)
    ws = plan.workspace(dev)

    def fwd_bwd():
        u = u0.detach().requires_grad_(True)
        loss = ag.masked_reconstruction_loss(u, plan, mask)
        loss.backward()

    plain = lambda: (plan.decompose(u0, ws, stream), plan.recompose(u0, ws, stream))
    for _ in range(3):
        fwd_bwd()
        plain()
    ms = _timed(torch, stream, fwd_bwd, 5)
    ms_plain = _timed(torch, stream, plain, 5)
    out = {"ms_per_step": ms, "plain_dec_rec_ms": ms_plain, "ratio_vs_2x_plain": ms / (2 * ms_plain),
           "workload": "257^3 FP32 masked reconstruction loss, forward + backward (adjoint kernels)"}
    plan.close()
    return out


def run_progressive(torch, mgard, plan, u, ws, stream, peak):
    """Recomposition of the 513^3 FP32 field from its first L and L-1
    coefficient classes (the finest one or two classes left out) against the
    full recomposition.  Every call starts from the decomposed field,
    restored by a device copy outside the call's events (median of 7).  The
    kernel that writes the finest grid (k_prolong) is timed by the plan's
    event pairs against the HBM roofline: it writes every finest node and
    reads the level-k values once."""
    import numpy as np

    L, S = plan.levels, 4
    plan.decompose(u, ws, stream)
    coef = u.clone()

    def median_call(fn, reps=7):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            u.copy_(coef)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sorted(a.elapsed_time(b) for a, b in ev)[reps // 2]

    for _ in range(3):
        u.copy_(coef)
        plan.recompose_classes(u, L, ws, stream)
    full = median_call(lambda: plan.recompose(u, ws, stream))
    rows = []
    for nc in (L, L - 1):
        ms = median_call(lambda: plan.recompose_classes(u, nc, ws, stream))
        mgard.mgard_profile_enable(plan.handle, 1)
        mgard.mgard_profile_read(plan.handle)
        median_call(lambda: plan.recompose_classes(u, nc, ws, stream), 3)
        prof = mgard.mgard_profile_read(plan.handle)
        mgard.mgard_profile_enable(plan.handle, 0)
        c, t = [(c, t) for k, lv, c, t in prof if k == 10][0]
        D = L + 1 - nc
        kb = int(np.prod(SHAPE)) * S + level_nodes(SHAPE, L)[D] * S
        per = t / c
        rows.append({"nclasses": nc, "dropped_levels": D, "ms": ms, "speedup_vs_full_recompose": full / ms,
                     "prolong_ms": per, "prolong_bytes": kb, "prolong_gbs": kb / (per / 1e3) / 1e9,
                     "prolong_frac_of_measured_hbm": kb / (per / 1e3) / 1e9 / peak})
    u.copy_(coef)
    plan.recompose(u, ws, stream)
    torch.cuda.synchronize()
    del coef
    return {"workload": "513^3 FP32 recomposition from the first L and L-1 of L+1 coefficient classes",
            "full_recompose_ms": full, "runs": rows}


def run_nonuniform(torch, mgard, synth, dev, stream, rank, world, max_over_ranks, uniform_ms):
    """513^3 FP32 on a tanh-clustered grid along every dimension
    (boundary-layer grading, beta = 2: spacings from 0.15x to 2.1x the mean):
    the same kernels with per-node interpolation, stencil and factor tables
    in place of the uniform fast paths; whole-job GB/s of the same
    algorithmic bytes, against the uniform step."""
    n = SHAPE[0]
    t = np.linspace(-1.0, 1.0, n)
    x = 0.5 * (1.0 + np.tanh(2.0 * t) / np.tanh(2.0))
    plan = mgard.Plan(SHAPE, dtype="f32", coords=[x.copy() for _ in SHAPE])
    u = synth.sinusoid_field_torch(SHAPE, N_MODES, SEED + rank, dev, torch.float32)
    ws = plan.workspace(dev)
    step = lambda: (plan.decompose(u, ws, stream), plan.recompose(u, ws, stream))
    for _ in range(3):
        step()
    ms = max_over_ranks(_timed(torch, stream, step, 10))
    d, r = algorithmic_bytes(SHAPE, plan.levels, 4)
    out = {"value": job_gbs(d + r, 1, world, ms), "unit": "GB/s", "ms_per_step": ms,
           "uniform_ms_per_step": uniform_ms, "slowdown_vs_uniform": ms / uniform_ms,
           "workload": "513^3 FP32 decompose+recompose, tanh-clustered coordinates (beta 2) on every axis"}
    del u, ws
    plan.close()
    torch.cuda.empty_cache()
    return out


def run_mixed(torch, mgard, synth, dev, stream, rank, world, max_over_ranks):
    """1025 x 1025 x 513 FP32 field (12 modes + Gaussian blob) per rank, FP64
    solves and coarse-level accumulation, 9 levels; whole-job GB/s."""
    shape = (1025, 1025, 513)
    plan = mgard.Plan(shape, dtype="f32_mixed")
    u = synth.sinusoid_field_torch(shape, 12, 3 + rank, dev, torch.float32, blob=True)
    ws = plan.workspace(dev)
    step = lambda: (plan.decompose(u, ws, stream), plan.recompose(u, ws, stream))
    for _ in range(3):
        step()
    ms = max_over_ranks(_timed(torch, stream, step, 5))
    d, r = algorithmic_bytes(shape, plan.levels, 4)
    out = {"value": job_gbs(d + r, 1, world, ms), "unit": "GB/s", "ms_per_step": ms, "levels": plan.levels,
           "workload": "1025x1025x513 FP32 field, FP64 solves and coarse arrays"}
    del u, ws
    plan.close()
    torch.cuda.empty_cache()
    return out


def run_case(spec):
    """One profiling case (no timing): --case SHAPE DTYPE REPS [NCLASSES] [TUNE]
    runs REPS decompose + recompose pairs of the seeded field of SHAPE
    (comma-separated sides) in DTYPE (f32 | f64 | f32_mixed); NCLASSES > 0
    rebuilds from that many coefficient classes; TUNE = param:value[,...]
    plan-wide tuning switches (mgard_plan_tune on level 0).  Prints one
    line, for runs under a profiler."""
    import torch

    from paper_2007_04457_gb300 import mgard, synth

    shape = tuple(int(x) for x in spec[0].split(","))
    dtype = spec[1] if len(spec) > 1 else "f32"
    reps = int(spec[2]) if len(spec) > 2 else 1
    nclasses = int(spec[3]) if len(spec) > 3 else 0
    plan = mgard.Plan(shape, dtype=dtype)
    if len(spec) > 4 and spec[4]:
        for kv in spec[4].split(","):
            k, v = kv.split(":")
            plan.tune(0, int(k), int(v))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u = synth.sinusoid_field_torch(shape, N_MODES if len(shape) == 3 else 8, SEED, "cuda", tdt)
    ws = plan.workspace(u.device)
    for _ in range(reps):
        plan.decompose(u, ws)
        if nclasses > 0:
            plan.recompose_classes(u, nclasses, ws)
        else:
            plan.recompose(u, ws)
    torch.cuda.synchronize()
    print(f"case ok: shape={shape} dtype={dtype} levels={plan.levels} reps={reps}"
          + (f" nclasses={nclasses}" if nclasses > 0 else ""))


def main():
    if "--case" in sys.argv:
        return run_case(sys.argv[sys.argv.index("--case") + 1:])
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-progressive", action="store_true")
    ap.add_argument("--no-nonuniform", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_2007_04457_gb300 import mgard, synth

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        dist_barrier(world)

    def max_over_ranks(x):
        return dist_max(x, world, dev)

    plan = mgard.Plan(SHAPE, dtype="f32")
    L = plan.levels
    S = 4
    u = synth.sinusoid_field_torch(SHAPE, N_MODES, SEED + rank, dev, torch.float32)
    ws = plan.workspace(dev)
    stream = torch.cuda.current_stream(dev)
    dec_b, rec_b = algorithmic_bytes(SHAPE, L, S)

    def step():
        plan.decompose(u, ws, stream)
        plan.recompose(u, ws, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # timed region: whole steps, with event pairs around the finest-level kernels
    mgard.mgard_profile_enable(plan.handle, 1)
    mgard.mgard_profile_read(plan.handle)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms)
    prof = [(KIND_NAMES[k], k, lv, c, t) for k, lv, c, t in mgard.mgard_profile_read(plan.handle)]
    mgard.mgard_profile_enable(plan.handle, 0)

    value = job_gbs(dec_b + rec_b, args.steps, world, ms)
    peak, peak_src = measured_peak()
    top = max(prof, key=lambda r: r[4]) if prof else None
    roof = None
    if top is not None:
        name, kind, lvl, c, t = top
        per_launch_ms = t / c
        kb = kernel_bytes(kind, SHAPE, S, S)
        achieved = kb / (per_launch_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": f"{name} (finest level)", "achieved": achieved,
                "peak": peak, "peak_source": f"{peak_src} hbm_gbs", "unit": "GB/s",
                "frac": achieved / peak, "traffic": recorded_traffic(name),
                "algorithmic_bytes_per_launch": kb, "ms_per_launch": per_launch_ms,
                "share_of_step": t / ms}

    finest_share = {f"{r[0]}": round(r[4] / ms, 4) for r in prof}

    # FP64 alongside (same workload in double precision)
    fp64 = None
    if not args.no_fp64:
        del u
        torch.cuda.empty_cache()
        plan64 = mgard.Plan(SHAPE, dtype="f64")
        u64 = synth.sinusoid_field_torch(SHAPE, N_MODES, SEED + rank, dev, torch.float64)
        ws64 = plan64.workspace(dev)
        for _ in range(3):
            plan64.decompose(u64, ws64, stream)
            plan64.recompose(u64, ws64, stream)
        torch.cuda.synchronize()
        k64 = max(3, args.steps // 4)
        e0.record(stream)
        for _ in range(k64):
            plan64.decompose(u64, ws64, stream)
            plan64.recompose(u64, ws64, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(e0.elapsed_time(e1))
        d64, r64 = algorithmic_bytes(SHAPE, L, 8)
        fp64 = {"value": job_gbs(d64 + r64, k64, world, ms64), "unit": "GB/s",
                "ms_per_step": ms64 / k64, "steps": k64}
        del u64, ws64, plan64
        torch.cuda.empty_cache()
        u = synth.sinusoid_field_torch(SHAPE, N_MODES, SEED + rank, dev, torch.float32)

    # end to end through the host-buffer entry points
    e2e = None
    if not args.no_e2e:
        # E2E_LANES fields in flight on as many streams (own device buffer,
        # workspace and host buffers each): one field's device-to-host copies
        # overlap another's host-to-device copies and compute.  Every step
        # still copies its input in from pinned host memory and its result
        # out.
        nbytes = u.numel() * S
        h_in = torch.empty(SHAPE, dtype=torch.float32, pin_memory=True)
        h_in.copy_(u.cpu())
        lanes = []
        for k in range(E2E_LANES):
            lanes.append({
                "u": u if k == 0 else torch.empty_like(u),
                "ws": ws if k == 0 else torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device=dev),
                "st": stream if k == 0 else torch.cuda.Stream(dev),
                "mid": torch.empty_like(h_in).pin_memory(),
                "out": torch.empty_like(h_in).pin_memory(),
            })

        def e2e_step(i):
            ln = lanes[i % E2E_LANES]
            st = ln["st"]
            wsb = ln["ws"].numel()
            mgard.mgard_decompose_host(plan.handle, h_in.data_ptr(), ln["mid"].data_ptr(), ln["u"].data_ptr(),
                                       ln["ws"].data_ptr(), wsb, st.cuda_stream)
            mgard.mgard_recompose_host(plan.handle, ln["mid"].data_ptr(), ln["out"].data_ptr(), ln["u"].data_ptr(),
                                       ln["ws"].data_ptr(), wsb, st.cuda_stream)

        def e2e_run(n):
            ev = torch.cuda.Event()
            ev.record(stream)
            for ln in lanes[1:]:
                ln["st"].wait_event(ev)
            for i in range(n):
                e2e_step(i)
            for ln in lanes[1:]:
                ev2 = torch.cuda.Event()
                ev2.record(ln["st"])
                stream.wait_event(ev2)

        e2e_run(2)
        torch.cuda.synchronize()
        ke = max(2 * E2E_LANES, args.steps // 4)
        barrier()
        e0.record(stream)
        e2e_run(ke)
        e1.record(stream)
        torch.cuda.synchronize()
        mse = max_over_ranks(e0.elapsed_time(e1))
        err = float((lanes[(ke - 1) % E2E_LANES]["out"] - h_in).abs().max() / h_in.abs().max())
        e2e = {"value": job_gbs(dec_b + rec_b, ke, world, mse), "unit": "GB/s",
               "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": 2 * nbytes,
               "ms_per_step": mse / ke, "steps": ke, "fields_in_flight": E2E_LANES, "round_trip_rel_err": err}

    # decomposition and recomposition timed separately (paper-style metric:
    # input bytes per second; the paper's pass model puts the attainable
    # rate at the measured single-pass bandwidth / 8.43 for 3D)
    ed0 = torch.cuda.Event(enable_timing=True)
    ed1 = torch.cuda.Event(enable_timing=True)
    t_dec = t_rec = 0.0
    for _ in range(5):
        ed0.record(stream)
        plan.decompose(u, ws, stream)
        ed1.record(stream)
        torch.cuda.synchronize()
        t_dec += ed0.elapsed_time(ed1)
        ed0.record(stream)
        plan.recompose(u, ws, stream)
        ed1.record(stream)
        torch.cuda.synchronize()
        t_rec += ed0.elapsed_time(ed1)
    t_dec, t_rec = max_over_ranks(t_dec / 5), max_over_ranks(t_rec / 5)
    in_bytes = int(np.prod(SHAPE)) * S
    paper_metric = {"decompose_input_gbs": in_bytes / (t_dec / 1e3) / 1e9,
                    "recompose_input_gbs": in_bytes / (t_rec / 1e3) / 1e9,
                    "decompose_ms": t_dec, "recompose_ms": t_rec,
                    "pass_model_peak_gbs": peak / 8.43,
                    "decompose_frac_of_pass_model": in_bytes / (t_dec / 1e3) / 1e9 / (peak / 8.43)}

    progressive = None if args.no_progressive else run_progressive(torch, mgard, plan, u, ws, stream, peak)
    nonuniform = None if args.no_nonuniform else run_nonuniform(
        torch, mgard, synth, dev, stream, rank, world, max_over_ranks, ms / args.steps)
    batched = None if args.no_batch else run_batched(torch, mgard, synth, dev, stream, rank)
    mixed = None if args.no_mixed else run_mixed(torch, mgard, synth, dev, stream, rank, world, max_over_ranks)
    adjoint = None if args.no_adjoint else run_adjoint(torch, mgard, synth, dev, stream, rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample()

    launches = (plan.launches(False) + plan.launches(True)) * args.steps
    if rank == 0:
        line = {
            "metric": "decompose+recompose GB/s (algorithmic bytes) at 513^3 FP32",
            "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: 12-mode sinusoid sum + N(0,1e-3) noise, seeded",
            "config": {"workload": "513^3 FP32 decompose+recompose, 9 levels, uniform grid",
                       "shape": list(SHAPE), "levels": L,
                       "l2": "inputs larger than L2 (540 MB field vs 129 MB L2), no flush",
                       "parallelism": f"independent fields, {world} GPU(s)"},
            "roofline": roof,
            "finest_level_kernel_share": finest_share,
            "fp64": fp64,
            "mixed": mixed,
            "batched": batched,
            "adjoint": adjoint,
            "progressive": progressive,
            "nonuniform": nonuniform,
            "paper_metric": paper_metric,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "gpu_launches": launches,
            "kernel_source": kernel_source_hash(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
