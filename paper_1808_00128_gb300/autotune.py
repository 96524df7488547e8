"""Launch-shape autotuner for the C library.

Times each candidate value of a context's launch knobs (lrs_set_tuning) on the
caller's actual workload with CUDA events and keeps the fastest.  Choices are
cached in a JSON file keyed by knob, register width n, padded term count and
batch size, so a later run with the same shapes reuses them without timing.
"""
from __future__ import annotations

import json
import os

CANDIDATES = {
    "amp_blocks_per_sm": [2, 4, 8, 16, 32],
    "norm_max_tiles": [256, 512, 1024, 2048, 4096],
    # fewer than 32 chains per block re-read each term's scalars (44 bytes) for too few
    # chains; the knob itself accepts 1..64
    "mc_chains_per_block": [32, 64],
    "norm_max_folds": [-1, 4, 8, 12],
    "mc_stages": [1, 2, 3, 4],
    "mc_lookahead": [1, 2],
}


MARGIN = 0.03


def _time_ms(fn, reps: int = 3, flush=None) -> float:
    """Median of `reps` timed calls; with `flush` (a device buffer larger than L2) the
    buffer is rewritten before each call, outside the timed interval, so every call
    starts from a cold L2 as a step of a long job does."""
    import statistics
    import torch
    fn()                                   # warm-up (and any lazy set-up)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def _load(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def _save(path, cache):
    if path:
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def tune(sim, x=None, L: int | None = None, chains: int | None = None, cache_path: str | None = None,
         reps: int = 5, flush_l2: int = 256 << 20, timer=None) -> dict:
    """Pick the fastest knob values for the given workload and set them on `sim`.

    x: amplitude batch (CUDA int64 tensor); L: number of equatorial states for
    norm estimation; chains: the chain count (chains must already be
    initialised on `sim`); flush_l2: bytes of a buffer rewritten before every timed
    call (0: time with a warm L2); timer: replaces the CUDA-event timing, a function
    of the job's callable returning milliseconds.  Returns {knob: (value, ms)}.
    """
    import torch
    cache = _load(cache_path)
    chosen = {}
    jobs = []
    flush = None
    if flush_l2 and timer is None:
        flush = torch.empty(flush_l2 // 4, dtype=torch.float32, device=f"cuda:{sim.device}")
    time_fn = timer if timer is not None else (lambda fn: _time_ms(fn, reps, flush))
    if x is not None:
        out = torch.empty((x.numel(), 2), dtype=torch.float64, device=x.device)
        jobs.append(("amp_blocks_per_sm", x.numel(), lambda: sim.amplitude(x, out=out)))
    if L:
        eta = torch.empty(L, dtype=torch.float64, device=f"cuda:{sim.device}")
        jobs.append(("norm_max_tiles", L, lambda: sim.norm_estimate(L, seed=1, eta=eta)))
        jobs.append(("norm_max_folds", L, lambda: sim.norm_estimate(L, seed=1, eta=eta)))
    if chains:
        jobs.append(("mc_chains_per_block", chains, lambda: sim.metropolis(16, seed=1)))
        jobs.append(("mc_stages", chains, lambda: sim.metropolis(16, seed=1)))
        jobs.append(("mc_lookahead", chains, lambda: sim.metropolis(16, seed=1)))
    for knob, batch, fn in jobs:
        key = f"{knob}|n={sim.n}|chi={sim.chi}|batch={batch}"
        if key in cache:
            sim.set_tuning(knob, cache[key]["value"])
            chosen[knob] = (cache[key]["value"], cache[key]["ms"])
            continue
        # the current value, if it is a candidate, is the incumbent; another candidate
        # must beat it by more than MARGIN (timing noise must not move a knob)
        cur = sim.get_tuning(knob)
        order = ([cur] if cur in CANDIDATES[knob] else []) + [v for v in CANDIDATES[knob] if v != cur]
        best = None
        for v in order:
            sim.set_tuning(knob, v)
            ms = time_fn(fn)
            if best is None or ms < best[1] * (1.0 - MARGIN):
                best = (v, ms)
        sim.set_tuning(knob, best[0])
        cache[key] = {"value": best[0], "ms": best[1]}
        chosen[knob] = best
    _save(cache_path, cache)
    return chosen
