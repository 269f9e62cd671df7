"""Rank-local steps of the sharded Algorithm 2 in plain numpy -- TEST INFRASTRUCTURE ONLY.

It drives ``paper_1708_04710_gb300.exchange.reduce_sharded`` over gloo ranks on the CPU, so
that the exchange protocol (which tables are merged, when, and which columns travel) can be
checked against the single-process oracle pass by pass. It holds the columns j = rank,
rank + k, rank + 2k, ... of a boundary matrix; beta, the dimensions, the pivot table (row ->
pivot column) and the essential estimate are replicated on every rank and updated from the
merged tables only. It shares no code with the oracle.

The rules follow the pass of Algorithm 2 (Phase 0 / I / II, Sec. 3), every decision taken
from the state at the start of the pass:
* empty active column -> final, positive;
* left-most for its low and low(j) = beta_j (Thm 5) -> pivot;
* left-most and no colliding column l < j of its dimension with low(l) >= low(j) (Phase I,
  Algorithm 5, Thms 6-7), tested as min{C(i') : i' >= low(j), dim i' = dim low(j)} > j with
  the merged collision table C -> pivot;
* Corollary 10 zero case: beta_j < 0 and every row of K_{d-1} up to low(j) in Paired -> zeroed;
  non-zero case: beta_j >= 0 and a single unpaired row of K_{d-1} in [beta_j, low(j)] -> that
  row is lowstar(j) (Lemma 9);
* clearing (Lemma 1): the column low(j) of every new pivot j is zeroed;
* Phase II: every other active column l with tab[low(l)] = s != l gets s added, unless s was
  zeroed by this pass (or is not a proven pivot, with strict = True, or its set is not acted
  on, with p < |C| sets, Sec. 3.4.1-3.4.2).
"""
from __future__ import annotations

import numpy as np

from paper_1708_04710_gb300.exchange import N_COUNTERS, NONE


def symmetric_difference(a, b):
    """a + b over F2 for sorted row lists, and the nontrivial scalar XORs |a u b| (Sec. 4.1)."""
    return np.setxor1d(a, b).astype(np.int32), len(np.union1d(a, b))


class CpuShard:
    def __init__(self, rank, world, colptr, rows, dim, beta, strict=False, cor10=True, sets=0,
                 priority=0):
        self.rank, self.world = rank, world
        self.m = m = len(dim)
        self.dim = np.asarray(dim, np.int64)
        self.beta = np.asarray(beta, np.int64)
        self.maxd = int(self.dim.max()) if m else 0
        # tables hold one entry per row that can be a low: the simplices below the top dimension
        self.row = np.nonzero(self.dim < self.maxd)[0]
        self.pos = np.full(max(m, 1), -1, np.int64)
        self.pos[self.row] = np.arange(len(self.row))
        self.n = len(self.row)
        self.strict, self.cor10, self.sets, self.priority = strict, cor10, sets, priority
        self.R = {int(j): np.asarray(rows[colptr[j]:colptr[j + 1]], np.int32)
                  for j in range(rank, m, world)}
        self.low = {j: int(c[-1]) if len(c) else -1 for j, c in self.R.items()}
        self.proven, self.final = set(), set()
        self.pred = {j: -1 for j in self.R}
        self.owner = np.full(m, -1, np.int64)  # replicated: row -> its proven pivot column
        self.in_E = np.ones(m, bool)            # replicated: E^l, starting from [m]
        self.st = np.zeros(N_COUNTERS, np.int64)

    def _active(self):
        return [j for j in self.R if j not in self.proven and j not in self.final]

    def _pivots(self):
        p = np.zeros(self.m, bool)
        p[self.owner[self.owner >= 0]] = True
        return p

    def leftmost_table(self):
        self.st[:] = 0
        t = np.full(self.n, NONE, np.int32)
        for j in self.R:  # ascending
            lo = self.low[j]
            if lo >= 0 and t[self.pos[lo]] == NONE:
                t[self.pos[lo]] = j
        return t

    def _tab(self, j):
        """The merged left-most column of column j's low."""
        return int(self.tab[self.pos[self.low[j]]])

    def collision_table(self, tab):
        self.tab = tab
        paired = self._pivots() | (self.beta >= 0) | (self.owner >= 0)
        self.unpaired = ~paired
        self.first_unpaired = [self.m] * (self.maxd + 1)
        for x in range(self.m - 1, -1, -1):
            if not paired[x]:
                self.first_unpaired[self.dim[x]] = x
        t = np.full(self.n, NONE, np.int32)
        for j in self._active():
            lo = self.low[j]
            if lo >= 0 and self._tab(j) != j and j < t[self.pos[lo]]:
                t[self.pos[lo]] = j
        return t

    def marks(self, collisions):
        dim, beta, st = self.dim, self.beta, self.st
        S = np.empty(self.n, np.int64)  # suffix minimum of C over the rows of each dimension
        run = [NONE] * (self.maxd + 1)
        for k in range(self.n - 1, -1, -1):
            d = dim[self.row[k]]
            run[d] = min(run[d], int(collisions[k]))
            S[k] = run[d]
        unpaired_rows = [np.nonzero(self.unpaired & (dim == d))[0] for d in range(self.maxd + 1)]
        self.new_pivots, self.zeroed = [], set()
        t = np.full(self.n, NONE, np.int32)
        for j in self._active():
            d, lo = int(dim[j]), self.low[j]
            st[0] += 1
            if lo < 0:
                self.zeroed.add(j)
                st[2] += 1
                continue
            if self._tab(j) == j and (lo == beta[j] or S[self.pos[lo]] > j):
                self.new_pivots.append(j)
                t[self.pos[lo]] = j
                st[1] += 1
            elif self.cor10 and d >= 1 and beta[j] < 0 and lo < self.first_unpaired[d - 1]:
                self.zeroed.add(j)
                st[3] += 1
            elif d >= 1 and beta[j] >= 0:
                # L_j: the unpaired rows of K_{d-1} in [beta_j, low(j)]
                u = unpaired_rows[d - 1]
                a, b = np.searchsorted(u, beta[j]), np.searchsorted(u, lo, side="right")
                if b == a:
                    st[10] += 1
                if b - a == 1 and self.pred[j] < 0:
                    self.pred[j] = int(u[a])
                    st[9] += 1
        return t

    def apply(self, new_pivots):
        rows = self.row[np.nonzero(new_pivots != NONE)[0]]
        self.owner[rows] = new_pivots[self.pos[rows]]
        self.proven.update(self.new_pivots)
        for i in rows:
            i = int(i)
            if i % self.world == self.rank:
                if i not in self.proven and i not in self.final:
                    self.st[4] += 1
                self.zeroed.add(i)
        for z in self.zeroed:
            if z not in self.final:
                self.final.add(z)
                self.R[z] = np.zeros(0, np.int32)
                self.low[z] = -1
        # E^l: drop Paired (after this pass's marks) and every low taken at the start of the pass
        self.in_E[self._pivots() | (self.beta >= 0) | (self.owner >= 0)] = False
        self.in_E[self.row[self.tab != NONE]] = False
        if self.rank == 0:
            self.st[8] = int(self.in_E.sum())
        flags = np.zeros(self.m, np.int32)
        flags[sorted(self.zeroed)] = 1
        return flags

    def _targets(self):
        return [(l, self._tab(l)) for l in self._active() if self._tab(l) != l]

    def set_sizes(self, zeroed):
        pivot = self._pivots()
        n = np.zeros((2, self.n), np.int64)
        for l, s in self._targets():
            if zeroed[s] or (self.strict and not pivot[s]):
                continue
            n[0, self.pos[self.low[l]]] += 1
            if self.beta[l] >= 0:
                n[1, self.pos[self.low[l]]] += 1
        return n

    def choose_sets(self, sizes):
        n, neg = sizes
        key = neg if self.priority == 1 else n
        order = sorted(np.nonzero(n > 0)[0], key=lambda k: (-key[k], -n[k], k))  # k: row order
        self.set_on = np.zeros(self.n, bool)
        self.set_on[np.asarray(order[:self.sets], np.int64)] = True

    def _eligible(self, l, s, pivot):
        if self.strict and not pivot[s]:
            return False
        return not self.sets or self.set_on[self.pos[self.low[l]]]

    def wanted_sources(self, additions):
        if not additions:
            return np.zeros(0, np.int64)
        pivot = self._pivots()
        want = {s for l, s in self._targets()
                if s % self.world != self.rank and self._eligible(l, s, pivot)}
        return np.array(sorted(want), np.int64)

    def serve(self, ids):
        lens, rows = [], []
        for s in ids:
            s = int(s)
            if s in self.zeroed:
                lens.append(-1)
            else:
                lens.append(len(self.R[s]))
                rows.append(self.R[s])
        return (np.array(lens, np.int64),
                np.concatenate(rows) if rows else np.zeros(0, np.int32))

    def add(self, fetched, additions):
        pivot = self._pivots()
        for l, s in self._targets():
            self.st[5] += 1
            if not additions or not self._eligible(l, s, pivot):
                continue
            if s % self.world == self.rank:
                src = None if s in self.zeroed else self.R[s]
            else:
                src = fetched.rows_of(s)
            if src is None:  # zeroed by this pass: the addition waits
                continue
            self.R[l], ops = symmetric_difference(self.R[l], src)
            self.low[l] = int(self.R[l][-1]) if len(self.R[l]) else -1
            self.st[6] += 1
            self.st[7] += ops

    def counters(self):
        return self.st.copy()

    def result(self):
        """Own columns: index -> (low, proven, predicted lowstar, reduced column)."""
        return {j: (self.low[j], j in self.proven, self.pred[j], self.R[j]) for j in self.R}
