"""Autotuner for steady windows: picks the tile and the launch shape (block
size, unroll, CTAs per SM) of a runtime context by timing one step of the
application on the device.

A *step* is a callable that issues the same steady work each time (one
in-place solver iteration of every problem of a batch, one sweep ...).  The
tuner changes the context's parameters between trials (dfs_set_launch_config
and the front end's tiling), so the stores, matrices and solver state stay
where they are: a trial advances the application's state, which the caller
resets afterwards.  The search is coordinate descent: each parameter in turn
takes the value of the fastest trial while the others stay fixed.  A
challenger replaces the incumbent only when it is faster by more than
`margin` (2 % by default, above the trial-to-trial noise of a few timed
steps; real differences between shapes are 5 % and more), so
candidates that tie within noise leave the starting setting in place and
repeated runs settle on the same kernels.

Tile and block size decide how reductions are split, so they fix the
rounding of a result; the chosen configuration is kept in a JSON cache (keyed
by the caller's workload key and the GPU name), so later runs reuse the same
choice instead of re-timing.
"""
from __future__ import annotations

import json
import math
import os
import time

from .binding import DfsError

# search order; a space names any subset.  tile: a fixed tile for every
# vector; tile_max: the cap of the size-dependent tile policy (tile None);
# rows: rows per point of 2-D and 3-D arrays
PARAMS = ("tile", "tile_max", "rows", "block", "unroll", "ctas_per_sm")
DEFAULT_SPACE = {"tile": [256, 512, 1024, 2048], "block": [128, 256, 512], "unroll": [1, 2, 4],
                 "ctas_per_sm": [0, 1, 2]}


def current(rt, params=("tile", "block", "unroll", "ctas_per_sm")) -> dict:
    return {p: getattr(rt, p) for p in params}


def apply(rt, cfg: dict) -> None:
    if (("tile" in cfg and cfg["tile"] != rt.tile) or ("tile_max" in cfg and cfg["tile_max"] != rt.tile_max)
            or ("rows" in cfg and cfg["rows"] != rt.rows)):
        rt.set_tiling(cfg.get("tile", rt.tile), cfg.get("rows", rt.rows), tile_max=cfg.get("tile_max"))
    rt.set_launch(cfg.get("block", rt.block), cfg.get("unroll", rt.unroll), cfg.get("ctas_per_sm", rt.ctas_per_sm))


def _kernel_ms(st: dict) -> float:
    return sum(v["ms"] for v in st.get("kernel_times", {}).values())


def measure(rt, step, warmup: int = 1, reps: int = 3) -> float:
    """Milliseconds per step: summed device time of the step's launches when
    the context times its launches, else host wall time to completion."""
    for _ in range(warmup):
        step()
    rt.sync()
    s0 = rt.stats()
    t0 = time.perf_counter()
    for _ in range(reps):
        step()
    rt.sync()
    wall = (time.perf_counter() - t0) * 1e3
    s1 = rt.stats()
    if s1.get("batch_fallbacks", 0) != s0.get("batch_fallbacks", 0):
        return math.inf                        # the candidate changed how the step runs
    dev = _kernel_ms(s1) - _kernel_ms(s0)
    return (dev if dev > 0 else wall) / reps


def tune(rt, step, space: dict | None = None, warmup: int = 1, reps: int = 3, key: str | None = None,
         cache_path: str | None = None, gpu: str = "", margin: float = 0.02) -> tuple[dict, list]:
    """Tunes rt for `step`; leaves rt configured with the best setting and
    returns (setting, trials) where trials is a list of (setting, ms)."""
    space = dict(space) if space else dict(DEFAULT_SPACE)
    params = [p for p in PARAMS if p in space]
    ck = f"{gpu}|{key}" if key else None
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if ck and ck in cache:
        best = cache[ck]["config"]
        apply(rt, best)
        return best, [(dict(t[0]), t[1]) for t in cache[ck]["trials"]]

    trials = []

    def trial(cfg):
        try:
            apply(rt, cfg)
            ms = measure(rt, step, warmup, reps)
        except DfsError:
            ms = math.inf                      # e.g. a block size whose kernel cannot be co-resident
            rt.sync_quiet()
        trials.append((dict(cfg), ms))
        return ms

    best = current(rt, params)
    best_ms = trial(best)
    for p in params:
        base = dict(best)
        for v in space[p]:
            if v == base[p]:
                continue
            cand = dict(base, **{p: v})
            ms = trial(cand)
            if ms < best_ms * (1.0 - margin):
                best, best_ms = cand, ms
    apply(rt, best)
    if ck and cache_path:
        cache[ck] = {"config": best, "ms": best_ms, "trials": [[c, (m if math.isfinite(m) else None)]
                                                               for c, m in trials]}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return best, trials
