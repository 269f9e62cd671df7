"""Autotuner for the Phase II addition kernel.

Six knobs shape the hot loop:
- ``staged_merge_max``: the longest merge that is still staged in shared memory (the threshold
  between the staged and the straight-from-memory merge);
- ``add_blocks_per_sm``: persistent blocks per SM (the grid shape);
- ``dense_threshold``: when a column's addition goes bit-packed (0 = as soon as the bitmap is
  the smaller form and the sum exceeds 32 rows, -1 = never, t > 0 = beyond max(bitmap words + 1,
  t) rows), the row-list to bitmap switch;
- ``warp_chunks_below``: the active-list length below which a warp, not a block, claims a chunk
  of the work queue (0 = 4,194,304, -1 = never), the block shape of the work queue;
- ``lane_merge_words``: the mean job length (target + source rows) up to which each lane merges
  its own job, before the lanes share every job's merge pieces (0 = 20, -1 = pieces throughout);
- ``narrow_chunks_below``: the active-list length below which the warps take chunks of 8 columns
  in the last passes (0 = 16 per warp of the grid, -1 = never).
The tuner times full reductions of the caller's own filtration, one knob at a time (coordinate
descent from the library defaults), and caches the winner per GPU model and workload class in a
JSON file (``$PH_GB300_CACHE`` or ``~/.cache/ph_gb300/autotune.json``). Every option gives the
same results; only the time differs.
"""
from __future__ import annotations

import json
import math
import os
import time
from pathlib import Path

from .native import Context

KNOBS = {
    "staged_merge_max": (1024, 512, 256),
    "add_blocks_per_sm": (4, 3, 2),
    "dense_threshold": (0, -1, 128, 1024),
    "warp_chunks_below": (0, -1, 1 << 20, 1 << 24),
    "lane_merge_words": (0, -1, 16, 40),
    "narrow_chunks_below": (0, -1, 1 << 18),
}
DEFAULTS = {"staged_merge_max": 1024, "add_blocks_per_sm": 4, "dense_threshold": 0,
            "warp_chunks_below": 0, "lane_merge_words": 0, "narrow_chunks_below": 0}


def cache_path() -> Path:
    p = os.environ.get("PH_GB300_CACHE")
    return Path(p) if p else Path.home() / ".cache" / "ph_gb300" / "autotune.json"


def load_cache(path: Path) -> dict:
    """The cached entries, or none when the file is missing or unreadable."""
    try:
        return json.loads(path.read_text())
    except (OSError, ValueError):
        return {}


def store_entry(path: Path, key: str, entry: dict) -> None:
    """Adds one entry to the cache file. The file is read again first, so entries that other
    processes stored meanwhile stay, and replaced in one rename, so no reader sees half of
    it."""
    path.parent.mkdir(parents=True, exist_ok=True)
    cache = load_cache(path)
    cache[key] = entry
    tmp = path.with_name(f"{path.name}.{os.getpid()}.tmp")
    tmp.write_text(json.dumps(cache, indent=1))
    os.replace(tmp, path)


def workload_key(gpu: str, m: int, max_dim: int, n_clouds: int) -> str:
    kind = "batched" if n_clouds > 1 else "single"
    return f"{gpu}|m2^{round(math.log2(max(m, 1)))}|dim{max_dim}|{kind}"


def _time_reduce(torch, coords, offsets, max_dim, max_diam2, opts, reps=2) -> float:
    ctx = Context(**opts)
    best = float("inf")
    for _ in range(reps + 1):
        ctx.build_filtration(coords, offsets, max_dim, max_diam2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.reduce()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    ctx.close()
    return best


def coordinate_descent(timer, knobs: dict, start: dict, verbose: bool = False):
    """Minimise timer(options) one knob at a time, keeping every improvement; returns (best
    options, best time, all trials)."""
    best = dict(start)
    best_t = timer(best)
    trials = [(dict(best), best_t)]
    for knob, values in knobs.items():
        for val in values:
            if val == best[knob]:
                continue
            cand = dict(best, **{knob: val})
            t = timer(cand)
            trials.append((cand, t))
            if verbose:
                print(f"autotune {cand} {1e3 * t:.2f} ms", flush=True)
            if t < best_t:
                best, best_t = cand, t
    return best, best_t, trials


def tune(coords, offsets=None, max_dim: int = 2, max_diam2: int = -1, use_cache: bool = True,
         verbose: bool = False) -> dict:
    """Best Context options for this filtration (cached per GPU model and workload class)."""
    import torch

    gpu = torch.cuda.get_device_name(coords.device)
    probe = Context()
    m = probe.build_filtration(coords, offsets, max_dim, max_diam2)
    nc = probe.n_clouds
    probe.close()
    key = workload_key(gpu, m, max_dim, nc)
    path = cache_path()
    if use_cache:
        # an entry tuned over other knob values (an older library) is tuned again
        opts = load_cache(path).get(key, {}).get("options")
        if opts and set(opts) == set(KNOBS) and all(opts[k] in v for k, v in KNOBS.items()):
            return dict(opts)
    best, best_t, trials = coordinate_descent(
        lambda o: _time_reduce(torch, coords, offsets, max_dim, max_diam2, o), KNOBS, DEFAULTS,
        verbose)
    if use_cache:
        store_entry(path, key, {"options": best, "ms": 1e3 * best_t,
                                "trials": [{"options": o, "ms": 1e3 * t} for o, t in trials]})
    return best
