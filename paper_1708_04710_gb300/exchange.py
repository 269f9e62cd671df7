"""One filtration reduced over several ranks: the per-pass exchange of Algorithm 2.

The columns of one boundary matrix are dealt round-robin by index over the ranks of a process
group: column j lives on rank j mod k, the non-contiguous distribution of columns the paper
argues for (Sec. 1, Sec. 3.4). Every pass of Algorithm 2 then needs the following traffic
between ranks, and nothing else:

1. ``tab``, the left-most column of every low, as an elementwise-min allreduce of the tables
   that each rank fills from its own columns.
2. Phase I (Algorithm 5, Thms 6-7) without a scan across ranks. Column j, left-most for its
   low, is proven when no colliding column l < j of its dimension has low(l) >= low(j). With
   C(i), the smallest colliding active column whose low is i, min-reduced over the ranks, that
   holds exactly when the minimum of C over the rows i' >= low(j) of low(j)'s dimension exceeds
   j. A suffix minimum on each rank then replaces the prefix-max scan over the whole filtration.
3. The new pivots, as an elementwise-min allreduce of their low -> column table. From it every
   rank updates its copy of the pivot table and of Paired (Sec. 3.2) and clears the columns it
   holds that are lows of new pivots (Lemma 1, clearing).
4. Phase II's source columns, fetched into local memory. Two all-to-alls send the request
   counts and the wanted column indices to the ranks that hold them, and two more return each
   column's length (-1 when this pass zeroed it, so the addition waits) and its rows.
5. The end of the loop: a pass without targets anywhere is the last (Sec. 2.3). That test
   rides on the next pass's first table as one more entry, so a pass takes three
   min-allreduces and four all-to-alls; the counters of every pass are summed once at the end.

With p < |C| processors (Sec. 3.4.1-3.4.2) the choice of the neighbour sets adds two
collectives: a max-allreduce of the columns zeroed by the pass and a sum-allreduce of the set
sizes, after which every rank orders the sets the same way.

A shard supplies the rank-local steps (the ``Shard`` protocol below); this module orders them
and moves their tables and columns. A table is an int32 array with one entry per row that can be
a low (the simplices below the top dimension, in filtration order: 80,200 of the 10.67 M
simplices of a 400-point Vietoris-Rips complex up to triangles), and ``NONE`` marks an empty
entry, so that an elementwise minimum merges tables. Collectives run on the tensors' own
device: CPU tensors over gloo, CUDA tensors over NCCL.
"""
from __future__ import annotations

import itertools
from typing import Protocol

import numpy as np

NONE = 2**31 - 1  # empty entry of a min-merged table
N_COUNTERS = 11   # per-pass counters, in the order of the reduction's pass statistics
TARGETS = 5       # the counter of colliding columns, whose sum ends the loop


class Shard(Protocol):
    """The rank-local steps of one pass, for the columns this rank holds."""

    def leftmost_table(self):
        """int32 table: the smallest own column of every low, NONE where no own column has
        it."""

    def collision_table(self, tab):
        """Takes the merged ``tab``. int32 table: the smallest own active column whose low is
        the row and that is not left-most for it (a colliding column), NONE where there is
        none."""

    def marks(self, collisions):
        """Takes the merged collision table. Applies Thm 5, Phase I, Corollary 10 and the
        empty-column rule to the own active columns; int32 table: the new pivots, low ->
        column."""

    def apply(self, new_pivots):
        """Takes the merged new-pivot table: updates the pivot table and clears. int32 [m], one
        entry per column: 1 for the own columns this pass zeroed, 0 elsewhere."""

    def set_sizes(self, zeroed):
        """Takes the merged zeroed flags. int64 [2, table]: per row i, the own targets of N(i)
        that this pass may reduce, and those of them known to be negative (Thm 5)."""

    def choose_sets(self, sizes) -> None:
        """Takes the merged set sizes and marks the sets that this pass acts on."""

    def wanted_sources(self, additions: bool):
        """int64, ascending: the other ranks' columns that this pass's additions use."""

    def serve(self, ids):
        """Own columns asked for: (int64 lengths, -1 for a column zeroed by this pass;
        int32 rows of the columns, concatenated in the order asked)."""

    def add(self, fetched: "Fetched", additions: bool) -> None:
        """Phase II on the own targets, with the other ranks' sources taken from ``fetched``."""

    def counters(self):
        """int64 [N_COUNTERS]: this rank's share of the pass counters."""


class Fetched:
    """Columns received from other ranks: ``rows_of(j)`` is None for a column zeroed by the
    pass that sent it."""

    def __init__(self, ids, lens, rows):
        self.ids = np.asarray(ids, np.int64)
        self.lens = np.asarray(lens, np.int64)
        self.rows = np.asarray(rows, np.int32)
        self.offsets = np.zeros(len(self.ids) + 1, np.int64)
        np.cumsum(np.maximum(self.lens, 0), out=self.offsets[1:])
        self._at = {int(j): k for k, j in enumerate(self.ids)}

    def __len__(self):
        return len(self.ids)

    def __contains__(self, j):
        return int(j) in self._at

    def rows_of(self, j):
        k = self._at[int(j)]
        if self.lens[k] < 0:
            return None
        return self.rows[self.offsets[k]:self.offsets[k + 1]]


class PassExchange:
    """The collectives of a pass over a process group, with the bytes this rank sends."""

    def __init__(self, group=None, device="cpu"):
        import torch
        import torch.distributed as dist

        self._torch, self._dist, self.group, self.device = torch, dist, group, device
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.table_bytes = 0
        self.column_bytes = 0

    def holder(self, j):
        """The rank that holds column j."""
        return j % self.world

    def _allreduce(self, a, op, dtype):
        t = self._torch.as_tensor(np.ascontiguousarray(a, dtype=dtype)).to(self.device)
        self._dist.all_reduce(t, op=op, group=self.group)
        self.table_bytes += t.numel() * t.element_size()
        return t.cpu().numpy()

    def min_merge(self, table):
        return self._allreduce(table, self._dist.ReduceOp.MIN, np.int32)

    def max_merge(self, table):
        return self._allreduce(table, self._dist.ReduceOp.MAX, np.int32)

    def sum_merge(self, values):
        return self._allreduce(values, self._dist.ReduceOp.SUM, np.int64)

    def _all_to_all(self, send, send_counts, recv_counts, dtype):
        torch = self._torch
        out = torch.empty(int(sum(recv_counts)), dtype=dtype, device=self.device)
        inp = torch.as_tensor(send).to(device=self.device, dtype=dtype)
        self._dist.all_to_all_single(out, inp, [int(c) for c in recv_counts],
                                     [int(c) for c in send_counts], group=self.group)
        self.column_bytes += inp.numel() * inp.element_size()
        return out.cpu().numpy()

    def fetch(self, wanted, serve) -> Fetched:
        """Columns ``wanted`` (indices held by other ranks) from their holders, each of which
        answers with ``serve``. Four all-to-alls: request counts, indices, lengths, rows."""
        torch = self._torch
        wanted = np.asarray(wanted, np.int64)
        dest = self.holder(wanted)
        order = np.argsort(dest, kind="stable")
        wanted = wanted[order]
        ask = np.bincount(dest, minlength=self.world).astype(np.int64)
        asked = self._all_to_all(ask, [1] * self.world, [1] * self.world, torch.int64)
        ids = self._all_to_all(wanted, ask, asked, torch.int64)
        lens, rows = serve(ids)
        lens = np.asarray(lens, np.int64)
        got_lens = self._all_to_all(lens, asked, ask, torch.int64)
        send_rows = [int(np.maximum(x, 0).sum()) for x in np.split(lens, np.cumsum(asked)[:-1])]
        recv_rows = [int(np.maximum(x, 0).sum())
                     for x in np.split(got_lens, np.cumsum(ask)[:-1])]
        got_rows = self._all_to_all(np.asarray(rows, np.int32), send_rows, recv_rows,
                                    torch.int32)
        return Fetched(wanted, got_lens, got_rows)


class ShardedResult(dict):
    """passes (the index of the last pass run), stats (one row of N_COUNTERS per pass run,
    summed over the ranks), exchange (bytes sent by all ranks per pass: tables, columns),
    converged."""

    def __getattr__(self, k):
        return self[k]


def reduce_sharded(shard: Shard, ex: PassExchange, max_passes: int = 100000,
                   sets: int = 0) -> ShardedResult:
    """Algorithm 2 pass by pass over the ranks of ``ex``; every rank calls it with its shard.

    A pass that finds no colliding column ends the loop (converged). After ``max_passes``
    passes with additions, one more pass applies its marks and clearing but no additions, as
    an early-stopped reduction does (Sec. 3.3). ``passes`` counts the passes that found
    collisions."""
    rows = []  # this rank's counters and bytes sent, one row per pass
    had_targets = True
    for p in itertools.count():
        additions = p < max_passes
        table = shard.leftmost_table()
        if p == 0:
            # every rank must hold tables of one length; all of them see the same answer
            lo, neg_hi = ex.min_merge(np.array([len(table), -len(table)], np.int32))
            if lo != -neg_hi:
                raise ValueError(f"ranks disagree on the table length ({lo} to {-neg_hi} rows)")
        # the left-most-column table carries one more entry, 1 on a rank whose previous pass
        # had no target: its minimum over the ranks is 1 when that pass was the last
        merged = ex.min_merge(np.append(table, np.int32(not had_targets)))
        if merged[-1]:
            rows[-1][N_COUNTERS] += ex.table_bytes
            break
        collisions = ex.min_merge(shard.collision_table(merged[:-1]))
        new_pivots = ex.min_merge(shard.marks(collisions))
        zeroed = shard.apply(new_pivots)
        if sets > 0 and additions:
            shard.choose_sets(ex.sum_merge(shard.set_sizes(ex.max_merge(zeroed))))
        shard.add(ex.fetch(shard.wanted_sources(additions), shard.serve), additions)
        counters = shard.counters()
        had_targets = counters[TARGETS] > 0
        rows.append(np.concatenate([counters, [ex.table_bytes, ex.column_bytes]]))
        ex.table_bytes = ex.column_bytes = 0
        if not additions:
            break
    total = ex.sum_merge(np.array(rows, np.int64))  # every pass's counters in one collective
    return ShardedResult(passes=len(rows) - 1, stats=total[:, :N_COUNTERS],
                         exchange=total[:, N_COUNTERS:],
                         converged=bool(total[-1, TARGETS] == 0))
