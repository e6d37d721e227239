"""Run decompose + recompose on a synthetic n^3 field, for use under a profiler.

    python -m paper_2007_04457_gb300.profile_case [n] [dtype] [reps] [ndim] [nclasses]

n: nodes per side (default 257), dtype: f32 | f64 | f32_mixed, reps: number of
decompose + recompose pairs, ndim: 1, 2 or 3 (default 3), nclasses: when
given, each recomposition rebuilds from the first nclasses coefficient
classes only.  Prints one line and exits 0; no timing is done here.
"""
import sys

import torch

from . import mgard, synth


def main(argv):
    n = int(argv[1]) if len(argv) > 1 else 257
    dtype = argv[2] if len(argv) > 2 else "f32"
    reps = int(argv[3]) if len(argv) > 3 else 2
    ndim = int(argv[4]) if len(argv) > 4 else 3
    nclasses = int(argv[5]) if len(argv) > 5 else 0
    shape = (n,) * ndim
    plan = mgard.Plan(shape, dtype=dtype)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    u = synth.sinusoid_field_torch(shape, 12, 2, "cuda", tdt)
    ws = plan.workspace(u.device)
    for _ in range(reps):
        plan.decompose(u, ws)
        if nclasses > 0:
            plan.recompose_classes(u, nclasses, ws)
        else:
            plan.recompose(u, ws)
    torch.cuda.synchronize()
    print(f"profile_case ok: shape={shape} dtype={dtype} levels={plan.levels} reps={reps}"
          + (f" nclasses={nclasses}" if nclasses > 0 else ""))


if __name__ == "__main__":
    main(sys.argv)
