"""Test-side checks that are independent of both the oracle and the CUDA path.

Nothing here reduces a boundary matrix the way the paper's algorithms do; these are the
textbook characterisations the tests pin the oracle against:

* GF(2) ranks by Gaussian elimination on Python-int bit rows.
* The pairing lemma through the rank function (Edelsbrunner-Harer, Computational Topology,
  VII.1): lowstar(j) = i iff r(i,j) - r(i+1,j) - r(i,j-1) + r(i+1,j-1) = 1, where r(a, b) is the
  rank of the lower-left block D[a:, :b+1].
* A reduction by randomly chosen left-to-right additions (any earlier column with the same low),
  whose low must agree with every other reduction (Sec. 2.3: lowstar does not depend on the
  reduction).
"""
from __future__ import annotations

import itertools
import random

import numpy as np


def dense_boundary(K) -> np.ndarray:
    m = K.m
    D = np.zeros((m, m), np.uint8)
    cp, rows = K["colptr"], K["rows"]
    for j in range(m):
        D[rows[cp[j]:cp[j + 1]], j] = 1
    return D


def anti_transpose(K):
    """J D^T J of the boundary matrix D of K, J reversing the index order: the coboundary matrix
    of the reversed filtration, as (dim, colptr, rows). It squares to zero and is graded by
    dim' = d_max - dim, so it is a boundary matrix in its own right."""
    dim, cp, rows = K["dim"], np.asarray(K["colptr"], np.int64), np.asarray(K["rows"], np.int64)
    m = len(dim)
    col = np.repeat(np.arange(m, dtype=np.int64), np.diff(cp))
    new_col, new_row = m - 1 - rows, m - 1 - col
    order = np.lexsort((new_row, new_col))
    colptr = np.zeros(m + 1, np.int64)
    colptr[1:] = np.cumsum(np.bincount(new_col, minlength=m))
    new_dim = (int(dim.max()) - np.asarray(dim)[::-1]).astype(np.int32)
    return (np.ascontiguousarray(new_dim), colptr,
            np.ascontiguousarray(new_row[order].astype(np.int32)))


def _insert(basis: dict, v: int) -> bool:
    while v:
        h = v.bit_length() - 1
        b = basis.get(h)
        if b is None:
            basis[h] = v
            return True
        v ^= b
    return False


def gf2_rank(M: np.ndarray) -> int:
    basis: dict = {}
    r = 0
    for row in np.asarray(M, np.uint8):
        v = int("".join("1" if x else "0" for x in row[::-1]) or "0", 2)
        r += _insert(basis, v)
    return r


def rank_pairing(D: np.ndarray) -> np.ndarray:
    """lowstar from the rank function alone (no column operations)."""
    m = D.shape[0]
    # r[a][b] for a in 0..m, b in -1..m-1 (stored at b+1)
    r = np.zeros((m + 1, m + 1), np.int64)
    row_bits = []
    for a in range(m):
        v = 0
        for j in np.nonzero(D[a])[0]:
            v |= 1 << int(j)
        row_bits.append(v)
    for b in range(m):
        mask = (1 << (b + 1)) - 1
        basis: dict = {}
        rank = 0
        for a in range(m - 1, -1, -1):
            rank += _insert(basis, row_bits[a] & mask)
            r[a, b + 1] = rank
    low = np.full(m, -1, np.int64)
    for j in range(m):
        for i in range(m):
            x = r[i, j + 1] - r[i + 1, j + 1] - r[i, j] + r[i + 1, j]
            if x == 1:
                low[j] = i
    return low


def random_reduction(D: np.ndarray, seed: int) -> np.ndarray:
    """Reduce by random valid left-to-right additions until low is injective."""
    rng = random.Random(seed)
    m = D.shape[0]
    cols = [set(np.nonzero(D[:, j])[0].tolist()) for j in range(m)]
    while True:
        by_low: dict = {}
        for j in range(m):
            if cols[j]:
                by_low.setdefault(max(cols[j]), []).append(j)
        pairs = [(a, b) for js in by_low.values() if len(js) > 1
                 for a, b in itertools.combinations(js, 2)]
        if not pairs:
            break
        j0, j = rng.choice(pairs)
        cols[j] ^= cols[j0]
    return np.array([max(c) if c else -1 for c in cols], np.int64)


def betti_by_rank(K) -> list:
    """b_p = dim C_p - rank d_p - rank d_{p+1} over F2 (Sec. 2.1)."""
    D = dense_boundary(K)
    dims = K["dim"]
    maxd = int(dims.max())
    ranks = {}
    for p in range(1, maxd + 1):
        cols = np.nonzero(dims == p)[0]
        rows = np.nonzero(dims == p - 1)[0]
        ranks[p] = gf2_rank(D[np.ix_(rows, cols)].T) if len(cols) and len(rows) else 0
    return [int((dims == p).sum()) - ranks.get(p, 0) - ranks.get(p + 1, 0)
            for p in range(maxd + 1)]


def closure(facets):
    out = set()
    for f in facets:
        f = tuple(sorted(f))
        for k in range(1, len(f) + 1):
            out.update(itertools.combinations(f, k))
    return out


def ordered_by_dim_lex(simplices):
    return sorted(simplices, key=lambda s: (len(s), s))


def random_compatible_order(simplices, seed: int):
    """A random filtration order: random values, each simplex above all its faces."""
    rng = random.Random(seed)
    val = {}
    for s in sorted(simplices, key=len):
        base = max((val[s[:k] + s[k + 1:]] for k in range(len(s))), default=0) if len(s) > 1 else 0
        val[s] = base + rng.randint(0, 3)
    return sorted(simplices, key=lambda s: (val[s], len(s), rng.random()))


def icosahedron_facets():
    phi = (1 + 5 ** 0.5) / 2
    V = []
    for a in (-1, 1):
        for b in (-1, 1):
            V += [(0, a, b * phi), (a, b * phi, 0), (b * phi, 0, a)]
    V = np.array(V)
    d = np.linalg.norm(V[:, None] - V[None], axis=2)
    adj = np.isclose(d, 2.0)
    return [t for t in itertools.combinations(range(12), 3)
            if adj[t[0], t[1]] and adj[t[0], t[2]] and adj[t[1], t[2]]]


# Phase II with p processors: seven vertices and nine edges in filtration order (the passes
# of this complex are derived by hand in test_oracle_pins.py)
BUDGET_EXAMPLE = [(v,) for v in range(7)] + [(0, 1), (0, 2), (0, 3), (0, 4), (1, 4), (2, 4),
                                            (3, 4), (0, 6), (5, 6)]


def cubical_grid(w, h, filled):
    """The cubical complex of a w x h grid of unit squares (vertices, edges, and the squares
    listed in `filled`), in a compatible order: boundary matrix columns of any length."""
    cells, index = [], {}

    def add(key, dim, faces):
        index[key] = len(cells)
        cells.append((dim, sorted(index[f] for f in faces)))

    for y in range(h + 1):
        for x in range(w + 1):
            add(("v", x, y), 0, [])
    for y in range(h + 1):
        for x in range(w):
            add(("h", x, y), 1, [("v", x, y), ("v", x + 1, y)])
    for y in range(h):
        for x in range(w + 1):
            add(("u", x, y), 1, [("v", x, y), ("v", x, y + 1)])
    for (x, y) in filled:
        add(("s", x, y), 2, [("h", x, y), ("h", x, y + 1), ("u", x, y), ("u", x + 1, y)])
    dims = np.array([c[0] for c in cells], np.int32)
    colptr = np.concatenate([[0], np.cumsum([len(c[1]) for c in cells])]).astype(np.int64)
    rows = np.array([r for c in cells for r in c[1]], np.int32)
    return dims, colptr, rows


def staircase(n):
    """Columns of dimension 1 over n + 1 rows (dimension 0) whose lows all meet at one row in
    every pass: column 1 = {n-1, n}, column j = {n-j, n} for j = 2..n. Pass k proves the
    left-most remaining column and adds it into every later one, which moves their common low
    down by one: n - 1 passes. Returns (dims, colptr, rows) for a general boundary load."""
    cols = [[n - 1, n]] + [[n - j, n] for j in range(2, n + 1)]
    dims = np.array([0] * (n + 1) + [1] * n, np.int32)
    lengths = np.cumsum([len(c) for c in cols])
    colptr = np.concatenate([[0] * (n + 2), lengths]).astype(np.int64)
    rows = np.array([r for c in cols for r in c], np.int32)
    return dims, colptr, rows
