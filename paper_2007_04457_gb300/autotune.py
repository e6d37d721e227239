"""Launch-shape autotuner.

Section III-C tunes thread-block sizes with a performance model that counts
memory transactions per configuration, then times only the best-ranked few
configurations.  This module does the same for the GB300 kernels:

* ``restriction_model`` estimates, for a tile height, the bytes the
  load-vector kernel moves at the finest level (every tile loads its rows
  plus a 3-row/4-column halo in whole 32-byte sectors, and the last tile of
  a dimension may be ragged), relative to the bytes of the field;
* ``tune`` ranks the tile configurations by that estimate, keeps the best
  ``top`` (three, as the paper does), times each of them with every solve
  warp count on the real plan, applies the fastest and caches it per
  (GPU, shape, dtype);
* ``tune_batch`` does the same for the persistent batch kernel: its
  launch parameters (blocks per SM, queue order) are ranked by the
  makespan of the library's list-scheduling model of the launch, and only
  the ``top`` best are timed.
"""
from __future__ import annotations

import json
import math
import os

CONFIGS = (0, 1, 2)                 # load-vector tile configurations the model ranks
DEFAULT = -1                        # each level keeps the plan's own choice (warp
                                    # strips where they apply), always timed
TILE_COLS = 64                      # coarse columns per tile
SOLVE_WARPS = (0, 8, 16)            # 0 = automatic
SECTOR = 32


def _tiles(m: int, t: int):
    """Sizes of the tiles along a dimension of m coarse nodes (the last tile
    takes the final node)."""
    if m <= 1:
        return [1]
    n = max(1, math.ceil((m - 1) / t))
    return [t] * (n - 1) + [m - t * (n - 1)]


def tile_rows(cfg: int, ndim: int, elem_bytes: int) -> int:
    """Coarse rows per tile of the load-vector kernel for configuration
    ``cfg`` (8, 4 or 16; the same for every dimension count and element
    size)."""
    return {0: 8, 1: 4, 2: 16}[cfg]


def restriction_model(shape, elem_bytes: int, cfg: int) -> float:
    """Estimated loaded bytes / field bytes of the finest-level restriction
    for tile configuration ``cfg`` (>= 1; smaller is better)."""
    shape = tuple(int(n) for n in shape if n > 1)
    if len(shape) == 1:
        return 1.0
    n1, n2 = shape[-2], shape[-1]
    m1, m2 = (n1 - 1) // 2 + 1, (n2 - 1) // 2 + 1
    rows = sum(2 * t + 3 for t in _tiles(m1, tile_rows(cfg, len(shape), elem_bytes)))
    cols_bytes = sum(math.ceil((2 * t + 8) * elem_bytes / SECTOR) * SECTOR for t in _tiles(m2, TILE_COLS))
    planes = shape[0] if len(shape) == 3 else 1
    loaded = rows * cols_bytes * planes
    return loaded / (n1 * n2 * planes * elem_bytes)


def ranked_configs(shape, elem_bytes: int, top: int = 3):
    """Tile configurations ordered by the model, best first, without
    configurations that give the same tile as a better one, cut to ``top``."""
    ndim = len([n for n in shape if int(n) > 1])
    order = sorted(CONFIGS, key=lambda c: (restriction_model(shape, elem_bytes, c), c))
    out, seen = [], set()
    for c in order:
        t = tile_rows(c, ndim, elem_bytes)
        if t not in seen:
            seen.add(t)
            out.append(c)
    return out[:top]


def _cache_path():
    return os.path.join(os.path.expanduser("~"), ".cache", "mgard_gb300", "tune.json")


def load_cache(path=None) -> dict:
    path = path or _cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path=None) -> None:
    path = path or _cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cache_key(gpu: str, shape, dtype: str) -> str:
    return f"{gpu}|{'x'.join(str(int(n)) for n in shape)}|{dtype}"


def apply(plan, cfg: int, warps: int) -> None:
    """Set the tile configuration and solve warps on every level of a plan
    (a configuration the device cannot run is skipped for that level;
    cfg = DEFAULT keeps each level's own choice)."""
    from .mgard import MgardError
    for level in range(plan.levels):
        if cfg != DEFAULT:
            try:
                plan.tune(level, 0, cfg)
            except MgardError:
                pass
        plan.tune(level, 1, warps)


def _time(plan, field, ws, reps: int) -> float:
    import torch
    for _ in range(2):
        plan.decompose(field, ws)
        plan.recompose(field, ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.decompose(field, ws)
        plan.recompose(field, ws)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(plan, field=None, top: int = 3, reps: int = 3, cache: bool = True, cache_path=None) -> dict:
    """Pick (tile config, solve warps) for ``plan`` by the model-pruned search
    (the plan's own per-level choice plus the ``top`` configurations of the
    byte model) and apply it.  ``field`` is a scratch tensor of the plan's shape and dtype
    (its contents are transformed back and forth); one is made if omitted.
    Returns {"cfg", "warps", "ms", "timed"}."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = cache_key(gpu, plan.shape, plan.dtype)
    store = load_cache(cache_path) if cache else {}
    if key in store:
        best = store[key]
        apply(plan, best["cfg"], best["warps"])
        return dict(best, cached=True)
    if field is None:
        field = torch.randn(plan.shape, dtype=plan.torch_dtype, device="cuda")
    ws = plan.workspace(field.device)
    elem = 8 if plan.dtype == "f64" else 4
    timed = []
    for cfg in [DEFAULT] + ranked_configs(plan.shape, elem, top):
        for warps in SOLVE_WARPS:
            try:
                apply(plan, cfg, warps)
                timed.append((_time(plan, field, ws, reps), cfg, warps))
            except Exception:
                continue
    ms, cfg, warps = min(timed)
    apply(plan, cfg, warps)
    best = {"cfg": cfg, "warps": warps, "ms": ms, "timed": len(timed)}
    if cache:
        store[key] = best
        save_cache(store, cache_path)
    return dict(best, cached=False)


BATCH_BLOCKS_PER_SM = (0, 1)        # 0 = as many as fit
BATCH_ORDERS = (0, 1)               # fields by size / longest remaining path first


def tune_batch(batch, fields, workspace, top: int = 2, reps: int = 2) -> dict:
    """Persistent batch kernel: rank (blocks per SM, queue order) by the
    modelled makespan of a decompose + recompose, time the ``top`` best on
    the real fields (decompose + recompose, which leaves them as they were up
    to rounding) and keep the fastest."""
    import torch

    if batch.get("eligible") != 1:
        return {"persistent": False}
    batch.tune(0, 1)
    cands = []
    for bps in BATCH_BLOCKS_PER_SM:
        for order in BATCH_ORDERS:
            batch.tune(3, bps)
            batch.tune(5, order)
            cands.append((batch.get("model_us_dec") + batch.get("model_us_rec"), bps, order))
    cands.sort()
    timed = []
    stream = torch.cuda.current_stream()
    for model_us, bps, order in cands[:max(1, top)]:
        batch.tune(3, bps)
        batch.tune(5, order)
        step = lambda: (batch.decompose(fields, workspace), batch.recompose(fields, workspace))
        step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        timed.append((e0.elapsed_time(e1) / reps, bps, order, model_us))
    ms, bps, order, model_us = min(timed)
    batch.tune(3, bps)
    batch.tune(5, order)
    return {"persistent": True, "blocks_per_sm": bps, "order": order, "ms": ms, "model_us": model_us,
            "ranked": [{"model_us": c[0], "blocks_per_sm": c[1], "order": c[2]} for c in cands],
            "timed": [{"ms": t[0], "blocks_per_sm": t[1], "order": t[2]} for t in timed]}
