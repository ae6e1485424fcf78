"""Autotuner for the launch shape of batches of graphs (bc_batch_set_tiles).

The tunable shape is (CTAs per SM of the per-vertex passes, of the rank-1 pass, of the
BC row sums, cap on accumulation CTAs per SM, the rank-1 pass's tile -- 16-byte vectors
per thread per work item, so its column chunk -- its schedule -- contiguous item
blocks per CTA or items dealt out in turn -- and the threads of an accumulation CTA,
512, 256 or 128).  The tuner runs coordinate descent from a
default: for each parameter in turn it applies one batch step with every candidate value
(each step consumes the next updates of the caller's stream, so the graphs advance as
they would anyway) and keeps the fastest.  Results are cached in
``_build/autotune.json`` next to the library, keyed by the batch's shape (number of
graphs, largest n rounded up to a power of two, distance type).
"""
from __future__ import annotations

import json
import os

from . import build as _build

DEFAULT = [4, 8, 8, 0, 4, 0, 256]
CANDIDATES = [[2, 4, 8], [4, 8, 16], [4, 8, 16], [0, 1], [1, 2, 4, 8], [0, 1], [512, 256, 128]]
CACHE = os.path.join(_build.BUILD, "autotune.json")
TIMED_STEPS = 2   # timed batch steps per candidate (after one untimed step that captures the graph)


def steps_needed() -> int:
    """Batch steps one tuning run consumes."""
    return (1 + TIMED_STEPS) * (1 + sum(len(c) - 1 for c in CANDIDATES))


def cache_key(count: int, n_max: int, dist: str) -> str:
    p = 1
    while p < n_max:
        p *= 2
    return f"G{count}-n{p}-{dist}"


def load_cache() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(key: str, tiles) -> None:
    data = load_cache()
    data[key] = list(int(t) for t in tiles)
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune(batch, next_step, key: str | None = None, use_cache: bool = True):
    """Tune ``batch`` (a binding.BCBatch).  ``next_step()`` returns the per-graph update
    lists of the next step.  Returns (tiles, trials) where trials lists (tiles, ms)."""
    if use_cache and key is not None:
        cached = load_cache().get(key)
        if cached and len(cached) == len(DEFAULT):
            batch.bc_batch_set_tiles(cached)
            return cached, []
    best = list(DEFAULT)
    trials = []

    def run(tiles):
        batch.bc_batch_set_tiles(tiles)
        rc, _ = batch.bc_batch_apply(next_step())   # captures a new CUDA graph, untimed
        if rc != 0:
            raise RuntimeError(f"batch step failed during tuning: {rc} {batch.last_error()}")
        ms = 0.0
        for _ in range(TIMED_STEPS):   # steps differ in work: more than one evens that out
            rc, _ = batch.bc_batch_apply(next_step())
            if rc != 0:
                raise RuntimeError(f"batch step failed during tuning: {rc} {batch.last_error()}")
            ms += batch.bc_batch_last_ms()
        trials.append((list(tiles), ms))
        return ms

    best_ms = run(best)
    for i, values in enumerate(CANDIDATES):
        incumbent = best[i]   # already timed: every other value of this parameter is run once
        for v in values:
            if v == incumbent:
                continue
            cand = list(best)
            cand[i] = v
            ms = run(cand)
            if ms < best_ms:
                best, best_ms = cand, ms
    batch.bc_batch_set_tiles(best)
    if key is not None:
        store(key, best)
    return best, trials
