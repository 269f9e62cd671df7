"""Sharding of the batched form over several GPUs.

Filtrations of different clouds are independent problems, so clouds are split across ranks
with no collective on the data path: longest-processing-time-first on an estimate of each
cloud's work (the number of simplices of dimension 0..max_dim, the sum of C(n, d + 1)), each
cloud to the currently lightest rank. Every rank computes the same assignment from the offsets alone.
"""
from __future__ import annotations

import heapq
import math

import numpy as np


def estimated_work(offsets, max_dim: int = 2) -> np.ndarray:
    n = np.diff(np.asarray(offsets, np.int64))
    return np.array([sum(math.comb(int(k), d + 1) for d in range(max_dim + 1)) for k in n],
                    np.float64)


def shard_clouds(offsets, world: int, max_dim: int = 2) -> list:
    """List of cloud indices (ascending) for every rank."""
    w = estimated_work(offsets, max_dim)
    order = sorted(range(len(w)), key=lambda c: (-w[c], c))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for c in order:
        load, r = heapq.heappop(heap)
        out[r].append(c)
        heapq.heappush(heap, (load + w[c], r))
    return [sorted(x) for x in out]


def local_batch(coords: np.ndarray, offsets, clouds: list):
    """Coordinates and offsets of a subset of the clouds, in the given order."""
    off = np.asarray(offsets, np.int64)
    parts = [coords[off[c]:off[c + 1]] for c in clouds]
    sizes = [len(p) for p in parts]
    loc_off = np.zeros(len(parts) + 1, np.int64)
    loc_off[1:] = np.cumsum(sizes)
    x = np.concatenate(parts) if parts else coords[:0]
    return np.ascontiguousarray(x), loc_off
