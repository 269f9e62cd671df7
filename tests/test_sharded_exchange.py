"""The single-filtration exchange over gloo ranks on the CPU.

One boundary matrix is dealt round-robin over 2, 3 and 4 ranks. Every rank runs
``exchange.reduce_sharded`` with the numpy shard of ``shard_cpu.py``, and the ranks meet only in
the protocol's collectives. The pass counters (all of them, pass by pass), the final low, the
proven pivots, the Corollary 10 predictions, the essential estimate and the reduced matrix R
must equal the single-process oracle's. That checks the tables the protocol merges: the
left-most columns, Phase I recast as a min-reduced collision table with a suffix minimum per
dimension, the new pivots and clearing, and the source columns fetched for Phase II.
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import pointclouds as pc
from helpers import closure, cubical_grid, random_compatible_order, staircase


def _general(orc, dims, cp, rows):
    m = len(dims)
    return orc.Complex(dim=np.asarray(dims, np.int32), diam2=np.zeros(m, np.int64),
                       verts=np.full((m, 4), -1, np.int32), colptr=np.asarray(cp, np.int64),
                       rows=np.asarray(rows, np.int32))


def _from_simplices(orc, simplices):
    index = {s: k for k, s in enumerate(simplices)}
    dims, cp, rows = [], [0], []
    for s in simplices:
        faces = sorted(index[s[:k] + s[k + 1:]] for k in range(len(s))) if len(s) > 1 else []
        dims.append(len(s) - 1)
        rows += faces
        cp.append(len(rows))
    return _general(orc, dims, cp, rows)


def _cases(orc):
    """(name, complex, options): Vietoris-Rips clouds, a random filtration of a closed
    surface, a cubical grid, the staircase, degenerate matrices, and the option grid of
    Algorithm 2."""
    vr3 = orc.vr_build(pc.random_cloud(13, 3, seed=21), 3)
    vr2 = orc.vr_build(pc.random_cloud(18, 3, seed=4), 2)
    ico = _from_simplices(orc, random_compatible_order(
        closure([(0, 1, 2), (0, 2, 3), (0, 3, 4), (0, 4, 1), (5, 1, 2), (5, 2, 3), (5, 3, 4),
                 (5, 4, 1)]), seed=3))
    grid = _general(orc, *cubical_grid(4, 3, [(x, y) for x in range(4) for y in range(3)
                                              if (x, y) != (1, 1)]))
    stair = _general(orc, *staircase(24))
    return [
        ("vr3", vr3, {}),
        ("vr3_strict", vr3, {"strict": True}),
        ("vr3_no_cor10", vr3, {"cor10": False}),
        ("vr3_stop2", vr3, {"max_passes": 2}),
        ("vr2", vr2, {}),
        ("vr2_sets5", vr2, {"sets": 5}),
        ("vr2_sets3_negative_first", vr2, {"sets": 3, "priority": 1}),
        ("octahedron", ico, {}),
        ("grid", grid, {}),
        ("staircase", stair, {}),
        # degenerate: no row can be a low (empty tables), and fewer columns than ranks' work
        ("vertices_only", _from_simplices(orc, [(v,) for v in range(5)]), {}),
        ("one_edge", _from_simplices(orc, [(0,), (1,), (0, 1)]), {}),
    ]


def _worker(rank, world, port, cases, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1708_04710_gb300.exchange import PassExchange, reduce_sharded
    from shard_cpu import CpuShard

    out = []
    for name, K, beta, opts in cases:
        sh = CpuShard(rank, world, K["colptr"], K["rows"], K["dim"], beta,
                      strict=opts.get("strict", False), cor10=opts.get("cor10", True),
                      sets=opts.get("sets", 0), priority=opts.get("priority", 0))
        res = reduce_sharded(sh, PassExchange(), max_passes=opts.get("max_passes", 100000),
                             sets=opts.get("sets", 0))
        out.append((name, dict(res), sh.result(), sh.in_E.copy()))
    q.put((rank, out))
    dist.destroy_process_group()


def _run_ranks(world, cases):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_worker, args=(r, world, port, cases, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return [got[r] for r in range(world)]


@pytest.mark.parametrize("world", [2, 3, 4])
def test_sharded_reduction_equals_oracle_pass_by_pass(orc, world):
    cases = [(name, K, orc.beta(K), opts) for name, K, opts in _cases(orc)]
    ranks = _run_ranks(world, cases)
    for c, (name, K, _, opts) in enumerate(cases):
        kw = dict(max_passes=opts.get("max_passes", 100000), strict=opts.get("strict", False),
                  cor10=opts.get("cor10", True), sets=opts.get("sets", 0),
                  priority=opts.get("priority", 0))
        ref = orc.reduce_pms(K, **kw)
        cp, rows = orc.reduce_pms_columns(K, **kw)
        results = [r[c] for r in ranks]
        for _, res, _, ess in results:
            # every rank sees the same merged counters and the same replicated E^l
            assert res["passes"] == ref.passes, name
            assert res["converged"] == ref.converged, name
            assert np.array_equal(res["stats"], ref.stats), name
            assert np.array_equal(ess, ref.ess_est), name
        cols = {}
        for _, _, own, _ in results:
            cols.update(own)
        assert sorted(cols) == list(range(K.m)), name
        for j in range(K.m):
            low, proven, pred, col = cols[j]
            assert low == ref.low[j], (name, j)
            assert proven == ref.proven[j], (name, j)
            assert pred == ref.predicted[j], (name, j)
            assert np.array_equal(col, rows[cp[j]:cp[j + 1]]), (name, j)
        # bytes moved: tables in every pass; a pass without targets fetches no column, so its
        # column exchange is the request counts alone (one int64 per pair of ranks)
        moved = results[0][1]["exchange"]
        assert moved.shape == (len(ref.stats), 2) and (moved[:, 0] > 0).all(), name
        if ref.converged:
            assert moved[-1, 1] == 8 * world * world, name


def _mismatch_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1708_04710_gb300.exchange import NONE, PassExchange, reduce_sharded

    class Lopsided:  # rank 1 counts one row more than rank 0
        def leftmost_table(self):
            return np.full(4 + rank, NONE, np.int32)

    try:
        reduce_sharded(Lopsided(), PassExchange())
        q.put((rank, "no error"))
    except ValueError as e:
        q.put((rank, str(e)))
    dist.destroy_process_group()


def test_ranks_with_unequal_tables_all_raise():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_mismatch_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == "ranks disagree on the table length (4 to 5 rows)"
