"""CUDA path against the CPU oracle, element by element, through the C ABI.

Everything is integer work, so every comparison is exact: the filtration (dimension, squared
diameter, vertex tuple), beta, the initial and final low, the persistence pairs, the essential
set and -- because every decision of a pass is taken from the pass's starting state -- the
per-pass counters of Algorithm 2 (pivots, zeroings, clearings, targets, additions, XORs).
"""
import hashlib
import json
import math
from pathlib import Path

import numpy as np
import pytest

import pointclouds as pc

pytestmark = pytest.mark.gpu
GOLDEN = Path(__file__).resolve().parent / "golden"


@pytest.fixture(scope="module")
def ph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_04710_gb300 import build

    build.build()
    import paper_1708_04710_gb300 as ph

    return ph


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build_lib()
    return oracle


def _gpu(ph, coords, max_dim, max_diam2=-1, offsets=None, **kw):
    import torch

    ctx = ph.Context(collect_stats=True, **kw)
    ctx.build_filtration(torch.from_numpy(np.ascontiguousarray(coords, np.int32)).cuda(),
                         offsets, max_dim, max_diam2)
    return ctx


def _check_counters(ctx, ref, cloud=0):
    """Per-pass counters and the essential estimate E^l against the oracle's pass loop."""
    ps = ctx.pass_stats()
    assert np.array_equal(ps[:, :8], ref.stats[:, :8])
    assert np.array_equal(ps[:, 9], ref.stats[:, 8])  # |E^l| after each pass's marks
    assert np.array_equal(ctx.essential_estimate(cloud), ref.ess_est)


def _canon(pairs_b, pairs_d, ess):
    p = np.stack([pairs_b, pairs_d], 1) if len(pairs_b) else np.zeros((0, 2), np.int64)
    o = np.lexsort((p[:, 0], p[:, 1])) if len(p) else np.zeros(0, int)
    return p[o].astype(np.int64), np.sort(np.asarray(ess, np.int64))


def _gpu_pairs(ctx, cloud):
    pr = ctx.pairs(cloud, on_device=False)
    es = ctx.essential(cloud, on_device=False)
    return {k: v.numpy() for k, v in pr.items()}, {k: v.numpy() for k, v in es.items()}


def _check_filtration(orc, ctx, cloud, K, low=None):
    f = ctx.filtration(cloud)
    assert np.array_equal(f["dim"], K["dim"])
    assert np.array_equal(f["diam2"], K["diam2"])
    vk = K["verts"].copy()
    assert np.array_equal(f["verts"], vk)
    assert np.array_equal(f["beta"], orc.beta(K))
    if low is not None:
        assert np.array_equal(f["low"], low)
    return f


def _check_reduced(orc, ctx, cloud, K, strict=False, cor10=True, stats=True):
    ref = orc.reduce_pms(K, strict=strict, cor10=cor10)
    assert ref.converged
    f = ctx.filtration(cloud)
    assert np.array_equal(f["low"], ref.low), "final low differs from the oracle"
    pr, es = _gpu_pairs(ctx, cloud)
    gp, ge = _canon(pr["birth"], pr["death"], es["idx"])
    op, oe = _canon(*orc.pairs_and_essential(ref.low, K["dim"])[0].T,
                    orc.pairs_and_essential(ref.low, K["dim"])[1])
    assert np.array_equal(gp, op)
    assert np.array_equal(ge, oe)
    # dims and diameters of the reported pairs / essentials
    d_by_idx = K["dim"]
    order = np.lexsort((pr["birth"], pr["death"]))
    assert np.array_equal(pr["dim"][order], d_by_idx[gp[:, 0]])
    assert np.array_equal(pr["birth_diam2"][order], K["diam2"][gp[:, 0]])
    assert np.array_equal(pr["death_diam2"][order], K["diam2"][gp[:, 1]])
    eo = np.argsort(es["idx"])
    assert np.array_equal(es["dim"][eo], d_by_idx[ge])
    assert np.array_equal(es["diam2"][eo], K["diam2"][ge])
    return ref


CASES = [
    ("gauss_3d_dim2", lambda: pc.random_cloud(24, 3, 1), 2, -1),
    ("gauss_2d_dim3", lambda: pc.random_cloud(14, 2, 2), 3, -1),
    ("gauss_5d_dim3_cut", lambda: pc.random_cloud(22, 5, 3), 3, int(6.0 * 65536 ** 2)),
    ("lattice_ties", lambda: pc.lattice_cloud(30, 2, 4, side=4), 2, -1),
    ("duplicates", lambda: np.repeat(pc.random_cloud(9, 3, 5), 2, axis=0), 2, -1),
    ("circle40", pc.circle40, 2, -1),
    ("edges_only", lambda: pc.random_cloud(50, 2, 6), 1, -1),
    ("one_point", lambda: pc.random_cloud(1, 3, 7), 2, -1),
    ("two_points", lambda: pc.random_cloud(2, 3, 8), 2, -1),
    ("three_points", lambda: pc.random_cloud(3, 3, 9), 3, -1),
    ("all_cut", lambda: pc.random_cloud(10, 3, 10), 2, 0),
    # dimensions 4 and 5 (six vertex slots of 8 bits); 15 points up to dimension 5 is the size
    # of the paper's ensembles (9,948 simplices)
    ("gauss_3d_dim4", lambda: pc.random_cloud(11, 3, 31), 4, -1),
    ("gauss_3d_dim5", lambda: pc.random_cloud(15, 3, 32), 5, -1),
    ("gauss_4d_dim5_cut", lambda: pc.random_cloud(16, 4, 33), 5, int(2.0 * 65536 ** 2)),
    ("lattice_dim4_ties", lambda: pc.lattice_cloud(14, 3, 34, side=3), 4, -1),
]


@pytest.mark.parametrize("name,gen,max_dim,cut", CASES, ids=[c[0] for c in CASES])
def test_filtration_and_reduction(ph, orc, name, gen, max_dim, cut):
    x = gen()
    K = orc.vr_build(x, max_dim, cut)
    ctx = _gpu(ph, x, max_dim, cut)
    assert ctx.m == K.m
    low0 = np.array([K["rows"][K["colptr"][j + 1] - 1] if K["colptr"][j + 1] > K["colptr"][j]
                     else -1 for j in range(K.m)], np.int32)
    _check_filtration(orc, ctx, 0, K, low0)
    st = ctx.reduce()
    assert st["converged"]
    ref = _check_reduced(orc, ctx, 0, K)
    assert st["passes"] == ref.passes
    _check_counters(ctx, ref)


@pytest.mark.parametrize("name,gen,max_dim,step,n_scales", [
    ("gaussian15_paper_grid", lambda: pc.ensemble15("gaussian15"), 5, 32768, 10),
    ("sphere_product15_paper_grid", lambda: pc.ensemble15("sphere_product15"), 5, 32768, 10),
    ("gauss_2d_coarse", lambda: pc.random_cloud(40, 2, 43), 2, 20000, 6),
    ("lattice_one_scale", lambda: pc.lattice_cloud(30, 2, 44, side=4), 3, 1 << 20, 1),
])
def test_scale_grid_filtration_and_reduction(ph, orc, name, gen, max_dim, step, n_scales):
    import torch

    x = gen()
    K = orc.vr_build(x, max_dim, scale_step=step, n_scales=n_scales)
    ctx = ph.Context(collect_stats=True)
    ctx.build_filtration_scales(torch.from_numpy(x).cuda(), None, max_dim, step, n_scales)
    assert ctx.m == K.m
    _check_filtration(orc, ctx, 0, K)
    for strict, cor10 in ((False, True), (True, False)):
        ctx2 = ph.Context(collect_stats=True, strict_phase2=strict, use_cor10=cor10)
        ctx2.build_filtration_scales(torch.from_numpy(x).cuda(), None, max_dim, step, n_scales)
        st = ctx2.reduce()
        ref = _check_reduced(orc, ctx2, 0, K, strict=strict, cor10=cor10)
        assert st["passes"] == ref.passes
        _check_counters(ctx2, ref)


@pytest.mark.parametrize("strict,cor10", [(True, True), (False, False), (True, False)])
def test_modes(ph, orc, strict, cor10):
    x = pc.random_cloud(40, 3, 11)
    K = orc.vr_build(x, 2)
    ctx = _gpu(ph, x, 2, strict_phase2=strict, use_cor10=cor10)
    st = ctx.reduce()
    ref = _check_reduced(orc, ctx, 0, K, strict=strict, cor10=cor10)
    assert st["passes"] == ref.passes
    _check_counters(ctx, ref)


@pytest.mark.parametrize("staged_max,items,bps", [(1, 4, 4), (16, 2, 1), (0, 1, 2), (0, 3, 3),
                                                  (0, 8, 4), (40, 8, 2), (0, 32, 4),
                                                  (100, 16, 1), (0, 0, 4), (0, 64, 3)])
def test_merge_paths_agree(ph, orc, staged_max, items, bps):
    # staged_max = 1: every merge from global memory; 16 / 40: mixed; 0: all staged
    x = pc.random_cloud(60, 3, 12)
    K = orc.vr_build(x, 2)
    ref = orc.reduce_pms(K)
    ctx = _gpu(ph, x, 2, staged_merge_max=staged_max, merge_items=items, add_blocks_per_sm=bps)
    ctx.reduce()
    assert np.array_equal(ctx.filtration(0)["low"], ref.low)
    assert np.array_equal(ctx.pass_stats()[:, :8], ref.stats[:, :8])


# bit-packed columns: small clouds built to high dimension have short row segments, so their
# columns fill in past the bitmap's size and additions run on bitmaps (dense + sparse and
# dense + dense); the results and every counter of Algorithm 2 stay the oracle's
DENSE_CASES = [
    ("gauss_3d_dim4", lambda: pc.random_cloud(11, 3, 31), 4, -1),
    ("gauss_2d_dim3", lambda: pc.random_cloud(14, 2, 2), 3, -1),
    ("gauss_3d_dim5", lambda: pc.random_cloud(15, 3, 32), 5, -1),
    ("lattice_dim4_ties", lambda: pc.lattice_cloud(14, 3, 34, side=3), 4, -1),
    ("circle40", pc.circle40, 2, -1),
    ("gauss_4d_dim5_cut", lambda: pc.random_cloud(16, 4, 33), 5, int(2.0 * 65536 ** 2)),
]


@pytest.mark.parametrize("threshold", [1, 0, 24])
@pytest.mark.parametrize("name,gen,max_dim,cut", DENSE_CASES, ids=[c[0] for c in DENSE_CASES])
def test_bit_packed_columns(ph, orc, name, gen, max_dim, cut, threshold):
    x = gen()
    K = orc.vr_build(x, max_dim, cut)
    packed = []
    for use_graph in (False, True):
        ctx = _gpu(ph, x, max_dim, cut, dense_threshold=threshold, use_graph=use_graph)
        st = ctx.reduce()
        assert st["converged"]
        ref = _check_reduced(orc, ctx, 0, K)
        assert st["passes"] == ref.passes
        _check_counters(ctx, ref)
        packed.append(ctx.pass_stats()[:, 12])
        assert packed[-1].sum() <= ref.stats[:, 6].sum()
    # the switch to bit-packing happens at the same pass in the graph and host-driven loops
    assert np.array_equal(packed[0], packed[1])
    if threshold == 1 and name in ("gauss_3d_dim4", "gauss_2d_dim3", "gauss_3d_dim5"):
        assert packed[0].sum() > 0, "no addition ran on bitmaps"


def test_bit_packed_columns_larger_complex(ph, orc):
    # 24 points to dimension 4 (55,454 simplices over several blocks): edge and triangle
    # segments are short enough that many columns go bit-packed, and bit-packed columns are
    # added to each other, moved, proven and cleared over many passes
    x = pc.random_cloud(24, 3, 77)
    K = orc.vr_build(x, 4)
    ref = orc.reduce_pms(K)
    ctx = _gpu(ph, x, 4, dense_threshold=1)
    st = ctx.reduce()
    assert st["passes"] == ref.passes
    assert np.array_equal(ctx.filtration(0)["low"], ref.low)
    _check_counters(ctx, ref)
    assert ctx.pass_stats()[:, 12].sum() > 0


@pytest.mark.parametrize("strict,cor10", [(True, True), (False, False)])
def test_bit_packed_columns_modes_and_batches(ph, orc, strict, cor10):
    import torch

    # a batch of clouds of different sizes (row segments, so bitmap sizes, differ per cloud)
    sizes = [9, 14, 3, 12, 1, 11]
    clouds = [pc.random_cloud(n, 3, 200 + i) for i, n in enumerate(sizes)]
    x = np.concatenate(clouds)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ctx = _gpu(ph, x, 4, offsets=off, dense_threshold=1, strict_phase2=strict, use_cor10=cor10)
    ctx.reduce()
    assert ctx.pass_stats()[:, 12].sum() > 0
    for c, xc in enumerate(clouds):
        _check_reduced(orc, ctx, c, orc.vr_build(xc, 4), strict=strict, cor10=cor10)
    # the paper's ensemble grid at dimension 5, partial and full
    xe = pc.ensemble15("sphere_product15")
    K = orc.vr_build(xe, 5, scale_step=32768, n_scales=10)
    for mp in (2, -1):
        cap = {} if mp < 0 else {"max_passes": mp}
        ref = orc.reduce_pms(K, strict=strict, cor10=cor10, **cap)
        ctx = ph.Context(collect_stats=True, strict_phase2=strict, use_cor10=cor10,
                         dense_threshold=1)
        ctx.build_filtration_scales(torch.from_numpy(xe).cuda(), None, 5, 32768, 10)
        ctx.reduce(max_passes=mp)
        assert np.array_equal(ctx.filtration(0)["low"], ref.low)
        _check_counters(ctx, ref)


@pytest.mark.parametrize("below", [-1, 1 << 30, 20000, 3000])
@pytest.mark.parametrize("use_graph", [False, True])
def test_chunk_shapes_agree(ph, orc, below, use_graph):
    # Phase II in 128-slot block chunks throughout (-1), 32-slot warp chunks throughout (2^30),
    # or switching from the first to the second mid-reduction (the active list drops below 20,000
    # or 3,000 columns); a batch of clouds, and a dense-mode run, switch too. Any job length
    # allows the switch here (warp_chunk_words = -1), so that these short jobs take it
    x = pc.random_cloud(60, 3, 12)
    K = orc.vr_build(x, 2)
    ref = orc.reduce_pms(K)
    ctx = _gpu(ph, x, 2, use_graph=use_graph, warp_chunks_below=below, warp_chunk_words=-1)
    st = ctx.reduce()
    assert st["passes"] == ref.passes
    assert np.array_equal(ctx.filtration(0)["low"], ref.low)
    _check_counters(ctx, ref)
    sizes = [17, 40, 5, 33]
    clouds = [pc.random_cloud(n, 3, 300 + i) for i, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ctx = _gpu(ph, np.concatenate(clouds), 2, offsets=off, use_graph=use_graph,
               warp_chunks_below=below // 2 if below > 0 else below, warp_chunk_words=-1)
    ctx.reduce()
    for c, xc in enumerate(clouds):
        _check_reduced(orc, ctx, c, orc.vr_build(xc, 2))
    xd = pc.random_cloud(11, 3, 31)
    Kd = orc.vr_build(xd, 4)
    refd = orc.reduce_pms(Kd)
    ctx = _gpu(ph, xd, 4, use_graph=use_graph, dense_threshold=1, warp_chunk_words=-1,
               warp_chunks_below=min(below, 2000) if below > 0 else below)
    ctx.reduce()
    assert np.array_equal(ctx.filtration(0)["low"], refd.low)
    _check_counters(ctx, refd)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_clouds(ph, orc, use_graph):
    sizes = [1, 2, 3, 17, 40, 5, 60, 33]
    clouds = [pc.random_cloud(n, 3, 100 + i) for i, n in enumerate(sizes)]
    x = np.concatenate(clouds)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ctx = _gpu(ph, x, 2, offsets=off, use_graph=use_graph)
    assert ctx.n_clouds == len(sizes)
    st = ctx.reduce()
    agg, ess = None, None
    for c, xc in enumerate(clouds):
        K = orc.vr_build(xc, 2)
        _check_filtration(orc, ctx, c, K)
        ref = _check_reduced(orc, ctx, c, K)
        assert np.array_equal(ctx.essential_estimate(c), ref.ess_est)
        s, e = ref.stats[:, :8], ref.stats[:, 8]
        if agg is None:
            agg, ess = s, e
        else:
            n = max(len(agg), len(s))
            agg = np.pad(agg, ((0, n - len(agg)), (0, 0))) + np.pad(s, ((0, n - len(s)), (0, 0)))
            # a converged cloud's estimate no longer changes
            ess = np.pad(ess, (0, n - len(ess)), mode="edge") + np.pad(e, (0, n - len(e)),
                                                                        mode="edge")
    assert np.array_equal(ctx.pass_stats()[:, :8], agg)
    assert np.array_equal(ctx.pass_stats()[:, 9], ess)
    assert st["passes"] == len(agg) - 1


@pytest.mark.parametrize("use_graph", [False, True])
def test_max_passes_partial_state(ph, orc, use_graph):
    x = pc.circle40()
    K = orc.vr_build(x, 2)
    for k in (0, 1, 3, 7):
        ctx = _gpu(ph, x, 2, use_graph=use_graph)
        st = ctx.reduce(max_passes=k)
        ref = orc.reduce_pms(K, max_passes=k)
        assert not st["converged"] and not ref.converged
        assert np.array_equal(ctx.filtration(0)["low"], ref.low)
        _check_counters(ctx, ref)  # E^l of the early-stopped reduction
        ctx.reset_reduction()
        st = ctx.reduce()
        assert st["converged"]
        _check_reduced(orc, ctx, 0, K)


@pytest.mark.parametrize("use_graph", [False, True])
def test_time_bound_stops_between_passes_and_resumes(ph, orc, use_graph):
    # a 1 ms bound stops the pass loop after some complete pass; every further call runs at
    # least one more pass and the result, pass count and counters are those of one call
    x = pc.torus400()[:160]
    K = orc.vr_build(x, 2)
    ref = orc.reduce_pms(K)
    ctx = _gpu(ph, x, 2, use_graph=use_graph, timeout_ms=1)
    timeouts = 0
    for _ in range(ref.passes + 2):
        try:
            st = ctx.reduce()
            break
        except ph.PHError as err:
            assert err.code == -5 and "time bound" in str(err)
            timeouts += 1
    else:
        pytest.fail("the reduction did not finish")
    assert timeouts >= 1
    assert st["converged"] and st["passes"] == ref.passes
    assert np.array_equal(ctx.filtration(0)["low"], ref.low)
    assert np.array_equal(ctx.pass_stats()[:, :8], ref.stats[:, :8])


@pytest.mark.parametrize("use_graph", [False, True])
def test_corollary10_predictions(ph, orc, use_graph):
    # the non-zero case of Corollary 10: the GPU predicts exactly the oracle's pairs, pass by
    # pass, and every prediction is a true pair of the finished reduction (Lemma 9)
    import torch

    cases = [(pc.random_cloud(40, 3, 109), 2, False, -1, 0),
             (pc.random_cloud(40, 3, 105), 2, True, -1, 0),
             (pc.ensemble15("trefoil15"), 5, False, 32768, 10), (pc.circle40(), 2, False, -1, 0)]
    for x, k, strict, step, ns in cases:
        K = (orc.vr_build(x, k, scale_step=step, n_scales=ns) if step > 0 else orc.vr_build(x, k))
        full = orc.reduce_pms(K, strict=strict)
        for mp in list(range(min(full.passes, 3))) + [-1]:
            ref = full if mp < 0 else orc.reduce_pms(K, max_passes=mp, strict=strict)
            ctx = ph.Context(collect_stats=True, strict_phase2=strict, predict_pairs=True,
                             use_graph=use_graph)
            xt = torch.from_numpy(x).cuda()
            if step > 0:
                ctx.build_filtration_scales(xt, None, k, step, ns)
            else:
                ctx.build_filtration(xt, None, k)
            ctx.reduce(max_passes=mp)
            pred = ctx.predicted_lows(0)
            assert np.array_equal(pred, ref.predicted)
            ps = ctx.pass_stats()
            assert np.array_equal(ps[:, 10], ref.stats[:, 9])
            assert not ps[:, 11].any()
            sel = pred >= 0
            assert np.array_equal(pred[sel], full.low[sel])


def test_triangulations(ph, orc):
    from helpers import closure, random_compatible_order

    data = json.loads((GOLDEN / "triangulations.json").read_text())
    data.pop("_about")
    for name, t in data.items():
        S = random_compatible_order(closure(t["facets"]), 5)
        K = orc.boundary_from_simplices(S)
        ctx = ph.Context(collect_stats=True)
        ctx.load_boundary(K["dim"], K["colptr"], K["rows"])
        ctx.reduce()
        es = ctx.essential(0, on_device=False)
        betti = np.bincount(es["dim"].numpy(), minlength=len(t["betti"])).tolist()
        assert betti == t["betti"], name
        ref = orc.reduce_pms(K)
        assert np.array_equal(ctx.filtration(0)["low"], ref.low), name
        assert np.array_equal(ctx.pass_stats()[:, :8], ref.stats[:, :8]), name


@pytest.mark.parametrize("kw", [{}, {"strict_phase2": True}, {"dense_threshold": 1},
                                {"warp_chunk_words": -1},
                                {"use_graph": False, "dense_threshold": -1,
                                 "warp_chunks_below": -1}])
def test_coboundary_matrix(ph, orc, kw):
    # The anti-transposed boundary matrix (the coboundary of the reversed filtration) loaded as
    # a general boundary: columns of up to n - 1 rows and an empty top-dimensional block. The
    # GPU reduces it to the oracle's lowstar pass by pass, and that lowstar mirrors the pairs
    # of the filtration itself (duality of persistent homology and cohomology).
    from helpers import anti_transpose

    for x, k in ((pc.random_cloud(40, 3, 600), 2), (pc.random_cloud(18, 3, 601), 4)):
        K = orc.vr_build(x, k)
        m = K.m
        dim, cp, rows = anti_transpose(K)
        Kc = orc.Complex(dim=dim, diam2=np.zeros(m, np.int64),
                         verts=np.full((m, 4), -1, np.int32), colptr=cp, rows=rows)
        ref = orc.reduce_pms(Kc, strict=kw.get("strict_phase2", False))
        ctx = ph.Context(collect_stats=True, **kw)
        ctx.load_boundary(dim, cp, rows)
        st = ctx.reduce()
        assert st["converged"] and st["passes"] == ref.passes
        low = ctx.filtration(0)["low"]
        assert np.array_equal(low, ref.low)
        assert np.array_equal(ctx.pass_stats()[:, :8], ref.stats[:, :8])
        low_k = orc.reduce_twist(K)[0]
        nz = np.nonzero(low >= 0)[0]
        mirror = np.full(m, -1, np.int32)
        mirror[m - 1 - low[nz]] = m - 1 - nz
        assert np.array_equal(mirror, low_k)


@pytest.mark.parametrize("sets,priority", [(1, 0), (1, 1), (3, 0), (7, 1), (10 ** 6, 0)])
def test_budgeted_phase2(ph, orc, sets, priority):
    # Phase II on p neighbour sets per pass (Sec. 3.4): the sets the GPU picks each pass are
    # the oracle's, so passes, every counter, E^l and the result agree exactly
    from helpers import BUDGET_EXAMPLE

    K0 = orc.boundary_from_simplices(BUDGET_EXAMPLE)
    ref = orc.reduce_pms(K0, sets=sets, priority=priority)
    ctx = ph.Context(collect_stats=True, phase2_sets=sets, phase2_priority=priority)
    ctx.load_boundary(K0["dim"], K0["colptr"], K0["rows"])
    st = ctx.reduce()
    assert st["passes"] == ref.passes
    assert np.array_equal(ctx.filtration(0)["low"], ref.low)
    assert np.array_equal(ctx.pass_stats()[:, :8], ref.stats[:, :8])
    for x, k in ((pc.random_cloud(30, 3, 500), 2), (pc.random_cloud(12, 3, 501), 4)):
        K = orc.vr_build(x, k)
        for strict in (False, True):
            ref = orc.reduce_pms(K, sets=sets, priority=priority, strict=strict)
            ctx = _gpu(ph, x, k, phase2_sets=sets, phase2_priority=priority,
                       strict_phase2=strict, use_graph=True)  # runs host-driven all the same
            st = ctx.reduce()
            assert st["passes"] == ref.passes
            _check_reduced(orc, ctx, 0, K, strict=strict)
            _check_counters(ctx, ref)


def test_budgeted_phase2_batched_and_partial(ph, orc):
    # a batch (one priority order over every cloud's sets) reaches each cloud's lowstar; an
    # early-stopped budgeted reduction is the oracle's state after the same passes
    sizes = [9, 20, 14]
    clouds = [pc.random_cloud(n, 3, 510 + i) for i, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ctx = _gpu(ph, np.concatenate(clouds), 3, offsets=off, phase2_sets=2, phase2_priority=1)
    ctx.reduce()
    for c, xc in enumerate(clouds):
        _check_reduced(orc, ctx, c, orc.vr_build(xc, 3))
    x = pc.circle40()
    K = orc.vr_build(x, 2)
    for mp in (1, 4, 9):
        ref = orc.reduce_pms(K, sets=5, priority=0, max_passes=mp)
        ctx = _gpu(ph, x, 2, phase2_sets=5)
        ctx.reduce(max_passes=mp)
        assert np.array_equal(ctx.filtration(0)["low"], ref.low)
        _check_counters(ctx, ref)
    with pytest.raises(ph.PHError):
        ph.Context(phase2_priority=2)


@pytest.mark.parametrize("use_graph", [False, True])
def test_capacity_growth_between_passes(ph, orc, use_graph):
    # one-word arenas: passes stop before any change, the host grows the arena and the pass
    # runs again; results, passes and counters are those of an unconstrained run
    x = pc.random_cloud(60, 3, 12)
    K = orc.vr_build(x, 2)
    ref = orc.reduce_pms(K)
    for extra in ({}, {"warp_chunks_below": 1 << 30, "warp_chunk_words": -1},
                  {"dense_threshold": 1}):
        ctx = _gpu(ph, x, 2, use_graph=use_graph, arena_words=1, **extra)
        st = ctx.reduce()
        assert st["passes"] == ref.passes
        _check_reduced(orc, ctx, 0, K)
        _check_counters(ctx, ref)


def test_allocation_failures_are_reported_and_resumable(ph, orc):
    # Allocation failures injected through the binding's allocator hook. Wherever a failure
    # hits -- the build, the reduction's set-up, or an arena grown between passes (one-word
    # arenas) -- the call returns PH_ERR_ALLOC without touching the GPU state it cannot
    # finish. Once allocations succeed again, the same calls resume and give the oracle's exact
    # reduction, counters included.
    import torch

    x = pc.random_cloud(60, 3, 12)
    K = orc.vr_build(x, 2)
    ref = orc.reduce_pms(K)
    xt = torch.from_numpy(x).cuda()

    def run(fail_at, use_graph):
        state = {"calls": 0, "fail": fail_at is not None, "where": None}

        def alloc(nbytes, stream):
            state["calls"] += 1
            if state["fail"] and state["calls"] > fail_at:
                return 0
            return torch.cuda.caching_allocator_alloc(nbytes, 0, stream)

        ctx = ph.Context(collect_stats=True, arena_words=1, use_graph=use_graph,
                         device_alloc=alloc, device_free=torch.cuda.caching_allocator_delete)
        for _ in range(2):
            try:
                if not ctx.m:
                    ctx.build_filtration(xt, None, 2)
                    state["built_at"] = state["calls"]
                st = ctx.reduce()
                state["reduced_at"] = state["calls"]
                break
            except ph.PHError as err:
                assert err.code == -2 and state["where"] is None, err
                state["where"] = "build" if not ctx.m else "reduce"
                state["fail"] = False
        assert st["converged"] and st["passes"] == ref.passes
        assert np.array_equal(ctx.filtration(0)["low"], ref.low)
        assert np.array_equal(ctx.pass_stats()[:, :8], ref.stats[:, :8])
        ctx.close()
        return state

    clean = run(None, True)
    n_build, n_all = clean["built_at"], clean["reduced_at"]
    assert n_all > n_build + 2  # the reduction allocates, and grows its arenas
    for use_graph in (True, False):
        seen = [run(k, use_graph)["where"] for k in
                (0, n_build // 2, n_build, n_build + 1, n_all - 2, n_all - 1)]
        assert seen[:2] == ["build", "build"] and set(seen[2:]) == {"reduce"}, seen


R_OPTS = [
    {},
    {"dense_threshold": 1},
    {"warp_chunks_below": 1 << 30, "warp_chunk_words": -1},
    {"staged_merge_max": 1},
    {"staged_merge_max": 16, "merge_items": 3},
    {"lane_merge_words": -1},
    {"lane_merge_words": 1 << 30},
    {"lane_merge_words": -1, "warp_chunks_below": 1 << 30, "warp_chunk_words": -1,
     "narrow_chunks_below": -1},
    {"lane_merge_words": -1, "warp_chunks_below": 1 << 30, "warp_chunk_words": -1,
     "narrow_chunks_below": 1 << 30, "dense_threshold": 1},
    {"strict_phase2": True},
    {"use_cor10": False},
    {"phase2_sets": 3, "phase2_priority": 1},
]


@pytest.mark.parametrize("opts", R_OPTS, ids=[",".join(o) or "default" for o in R_OPTS])
def test_reduced_matrix_equals_oracle(ph, orc, opts):
    # Every column of R, row by row, after complete and partial reductions: the column
    # additions themselves (register networks, staged and global merge paths, bitmaps, both
    # chunk shapes) against the oracle's sorted-array symmetric differences
    okw = {"strict": opts.get("strict_phase2", False), "cor10": opts.get("use_cor10", True),
           "sets": opts.get("phase2_sets", 0), "priority": opts.get("phase2_priority", 0)}
    cases = [(pc.random_cloud(24, 3, 1), 2), (pc.random_cloud(11, 3, 31), 4), (pc.circle40(), 2),
             (pc.random_cloud(60, 3, 12), 2)]
    for x, k in cases:
        K = orc.vr_build(x, k)
        for mp in (-1, 2):
            cp, rows = orc.reduce_pms_columns(K, **okw, **({} if mp < 0 else {"max_passes": mp}))
            ctx = _gpu(ph, x, k, **opts)
            ctx.reduce(max_passes=mp)
            gcp, grows = ctx.columns(0)
            assert np.array_equal(gcp, cp), (k, mp)
            assert np.array_equal(grows, rows), (k, mp)
    # a batch: each cloud's columns are those of the cloud reduced alone
    if not opts.get("phase2_sets"):
        sizes = [9, 20, 14]
        clouds = [pc.random_cloud(n, 3, 700 + i) for i, n in enumerate(sizes)]
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        ctx = _gpu(ph, np.concatenate(clouds), 3, offsets=off, **opts)
        ctx.reduce()
        for c, xc in enumerate(clouds):
            cp, rows = orc.reduce_pms_columns(orc.vr_build(xc, 3), **okw)
            gcp, grows = ctx.columns(c)
            assert np.array_equal(gcp, cp) and np.array_equal(grows, rows), c


def test_invalid_arguments(ph):
    import torch

    ctx = ph.Context()
    x = torch.zeros((4, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(ph.PHError):
        ctx.build_filtration(x, None, 6)  # max_dim out of range
    with pytest.raises(ph.PHError) as err:  # above dimension 3 a cloud holds at most 254 points
        ctx.build_filtration(torch.zeros((255, 3), dtype=torch.int32, device="cuda"), None, 4)
    assert err.value.code == -4
    with pytest.raises(ph.PHError):
        ctx.build_filtration(x, [0, 2, 3], 2)  # offsets must end at N
    big = torch.full((3, 2), 1 << 25, dtype=torch.int32, device="cuda")
    with pytest.raises(ph.PHError):
        ctx.build_filtration(big, None, 2)  # coordinates beyond the grid bound
    with pytest.raises(ph.PHError):
        ctx.reduce()  # no filtration
    ctx.build_filtration(x, None, 2)
    ctx.reduce()
    assert ctx.essential(0, on_device=False)["idx"].numel() == 2  # b0 = b2 = 1


# ------------------------------------------------------------------------------------------
# full-size workloads against stored oracle results (tests/golden/make_golden.py)
# ------------------------------------------------------------------------------------------
def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _golden(name):
    p = GOLDEN / f"{name}.json"
    if not p.exists():
        pytest.skip(f"{p.name} not generated")
    return json.loads(p.read_text())


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("name", ["circle40", "gauss8_120", "torus400"])
def test_full_size_single(ph, name, use_graph):
    g = _golden(name)
    x = {"circle40": pc.circle40, "gauss8_120": pc.gauss8_120, "torus400": pc.torus400}[name]()
    assert _sha(x) == g["coords_sha"], "generator drift: coordinates differ from the golden's"
    max_dim = 3 if name == "gauss8_120" else 2
    ctx = _gpu(ph, x, max_dim, g.get("max_diam2", -1), use_graph=use_graph)
    assert ctx.m == g["m"]
    st = ctx.reduce()
    assert st["converged"] and st["passes"] == g["passes"]
    assert np.array_equal(ctx.pass_stats()[:, :8], np.array(g["pass_stats"], np.int64))
    pr, es = _gpu_pairs(ctx, 0)
    gp, ge = _canon(pr["birth"], pr["death"], es["idx"])
    assert _sha(gp) == g["pairs_sha"]
    assert _sha(ge) == g["ess_sha"]
    assert np.bincount(es["dim"], minlength=max_dim + 1).tolist() == g["ess_per_dim"]


@pytest.mark.parametrize("narrow", [-1, 1 << 30])
def test_full_size_torus400_chunk_widths(ph, narrow):
    # the late passes in 32-slot warp chunks throughout (-1), or in 8-slot warp chunks from the
    # first pass with merge pieces on (2^30): the golden pairs and per-pass counters either way
    g = _golden("torus400")
    ctx = _gpu(ph, pc.torus400(), 2, narrow_chunks_below=narrow)
    st = ctx.reduce()
    assert st["converged"] and st["passes"] == g["passes"]
    assert np.array_equal(ctx.pass_stats()[:, :8], np.array(g["pass_stats"], np.int64))
    pr, es = _gpu_pairs(ctx, 0)
    gp, ge = _canon(pr["birth"], pr["death"], es["idx"])
    assert _sha(gp) == g["pairs_sha"] and _sha(ge) == g["ess_sha"]


@pytest.mark.parametrize("use_graph", [False, True])
def test_full_size_batch512(ph, use_graph):
    g = _golden("batch512")
    x, off = pc.batch512()
    assert _sha(x) == g["coords_sha"] and _sha(off) == g["offsets_sha"]
    ctx = _gpu(ph, x, 2, offsets=off, use_graph=use_graph)
    assert ctx.m == g["m"]
    st = ctx.reduce()
    assert st["converged"] and st["passes"] == g["passes"]
    assert np.array_equal(ctx.pass_stats()[:, :8], np.array(g["pass_stats"], np.int64))
    h = hashlib.sha256()
    for c in range(len(off) - 1):
        pr, es = _gpu_pairs(ctx, c)
        gp, ge = _canon(pr["birth"], pr["death"], es["idx"])
        h.update(gp.tobytes())
        h.update(ge.tobytes())
    assert h.hexdigest() == g["all_sha"]


def test_closed_form_complete_skeleton_large(ph):
    # b_2 of the complete 2-skeleton on n points is C(n-1, 3), at a size no oracle runs
    x = pc.to_grid(pc.sphere(160, pc.rng_for(9)))
    ctx = _gpu(ph, x, 2)
    assert ctx.m == 160 + math.comb(160, 2) + math.comb(160, 3)
    ctx.reduce()
    es = ctx.essential(0, on_device=False)
    assert np.bincount(es["dim"].numpy(), minlength=3).tolist() == [1, 0, math.comb(159, 3)]
    pr = ctx.pairs(0, on_device=False)
    assert np.all(pr["birth_diam2"].numpy() <= pr["death_diam2"].numpy())


@pytest.mark.parametrize("use_graph", [False, True])
def test_context_rebuilt_with_other_filtrations(ph, orc, use_graph):
    # one context: a batched filtration first, then single clouds of other sizes (once, freed
    # buffers of an earlier filtration were freed again after their addresses were reused)
    x, off = pc.batch512(n_clouds=48)
    ctx = _gpu(ph, x, 2, offsets=off, use_graph=use_graph)
    ctx.reduce()
    ctx.pairs(0)
    import torch

    for c in range(len(off) - 1):
        xc = x[off[c]:off[c + 1]]
        ctx.build_filtration(torch.from_numpy(np.ascontiguousarray(xc)).cuda(), None, 2)
        st = ctx.reduce()
        assert st["converged"]
        K = orc.vr_build(xc, 2)
        _check_reduced(orc, ctx, 0, K)


def test_autotuned_options_stay_exact(ph, orc, tmp_path, monkeypatch):
    import torch

    from paper_1708_04710_gb300 import autotune

    monkeypatch.setenv("PH_GB300_CACHE", str(tmp_path / "tune.json"))
    x = pc.random_cloud(70, 3, 21)
    opts = autotune.tune(torch.from_numpy(x).cuda(), None, 2)
    assert (tmp_path / "tune.json").exists()
    assert autotune.tune(torch.from_numpy(x).cuda(), None, 2) == opts  # from the cache
    K = orc.vr_build(x, 2)
    ctx = _gpu(ph, x, 2, **opts)
    ctx.reduce()
    _check_reduced(orc, ctx, 0, K)


def test_all_clouds_at_once(ph, orc):
    sizes = [12, 30, 7]
    clouds = [pc.random_cloud(n, 3, 200 + i) for i, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    ctx = _gpu(ph, np.concatenate(clouds), 2, offsets=off)
    ctx.reduce()
    allp = ctx.pairs(-1, on_device=False)
    alle = ctx.essential(-1, on_device=False)
    parts = [ctx.pairs(c, on_device=False) for c in range(3)]
    eparts = [ctx.essential(c, on_device=False) for c in range(3)]
    for k in ("birth", "death", "dim"):
        assert np.array_equal(allp[k].numpy(), np.concatenate([p[k].numpy() for p in parts]))
    assert np.array_equal(alle["idx"].numpy(), np.concatenate([e["idx"].numpy() for e in eparts]))


def test_random_complexes_and_options(ph, orc):
    # Seeded sweep: random small clouds (2-18 points, 1-4 coordinates, dimensions up to 5, with
    # or without a diameter cut) under random combinations of the options; each run must give
    # the oracle's lows, counters and reduced matrix, after a complete or a partial reduction
    import torch

    rng = np.random.default_rng(1708)
    for case in range(200):
        n = int(rng.integers(2, 19))
        dim_cap = 5 if n <= 12 else (4 if n <= 15 else 3)
        k = int(rng.integers(1, min(dim_cap, n - 1) + 1)) if n > 2 else 1
        x = pc.random_cloud(n, int(rng.integers(1, 5)), 900 + case)
        cut = -1
        if rng.random() < 0.3:
            d2 = ((x[:, None, :].astype(np.int64) - x[None, :, :]) ** 2).sum(-1)
            cut = int(np.quantile(d2[np.triu_indices(n, 1)], rng.uniform(0.2, 0.9)))
        opts = {}
        if rng.random() < 0.3:
            opts["dense_threshold"] = int(rng.choice([1, 8, 24]))
        if rng.random() < 0.3:
            opts.update(warp_chunks_below=1 << 30, warp_chunk_words=-1)
        if rng.random() < 0.3:
            opts["staged_merge_max"] = int(rng.choice([1, 6, 40]))
            opts["merge_items"] = int(rng.choice([0, 2, 5, 16]))
        if rng.random() < 0.4:
            opts["lane_merge_words"] = int(rng.choice([-1, 4, 12, 1 << 30]))
        if rng.random() < 0.3:
            opts["narrow_chunks_below"] = int(rng.choice([-1, 50, 1 << 30]))
        if rng.random() < 0.25:
            opts["strict_phase2"] = True
        if rng.random() < 0.2:
            opts["use_cor10"] = False
        if rng.random() < 0.2:
            opts.update(phase2_sets=int(rng.integers(1, 6)),
                        phase2_priority=int(rng.integers(0, 2)))
        opts["use_graph"] = bool(rng.random() < 0.6)
        mp = -1 if rng.random() < 0.7 else int(rng.integers(0, 4))
        okw = {"strict": opts.get("strict_phase2", False), "cor10": opts.get("use_cor10", True),
               "sets": opts.get("phase2_sets", 0), "priority": opts.get("phase2_priority", 0)}
        if mp >= 0:
            okw["max_passes"] = mp
        K = orc.vr_build(x, k, cut)
        ref = orc.reduce_pms(K, **okw)
        cp, rows = orc.reduce_pms_columns(K, **okw)
        ctx = ph.Context(collect_stats=True, **opts)
        ctx.build_filtration(torch.from_numpy(x).cuda(), None, k, cut)
        st = ctx.reduce(max_passes=mp)
        where = (case, n, k, cut, mp, opts)
        assert st["passes"] == ref.passes, where
        assert np.array_equal(ctx.filtration(0)["low"], ref.low), where
        assert np.array_equal(ctx.pass_stats()[:, :8], ref.stats[:, :8]), where
        gcp, grows = ctx.columns(0)
        assert np.array_equal(gcp, cp) and np.array_equal(grows, rows), where
        ctx.close()


def test_random_batches_grids_and_predictions(ph, orc):
    # Seeded sweep over what the first sweep keeps fixed: batches of random clouds (each cloud
    # against the oracle run on it alone), the scale-grid build, Corollary 10 predictions and
    # the essential estimate of early-stopped reductions
    import torch

    rng = np.random.default_rng(4710)
    for case in range(60):
        nb = int(rng.integers(1, 6))
        sizes = [int(rng.integers(1, 15)) for _ in range(nb)]
        D = int(rng.integers(1, 4))
        k = int(rng.integers(1, 4))
        clouds = [pc.random_cloud(n, D, 2000 + 10 * case + i) for i, n in enumerate(sizes)]
        opts = {"use_graph": bool(rng.random() < 0.5), "predict_pairs": bool(rng.random() < 0.5)}
        if rng.random() < 0.3:
            opts["dense_threshold"] = 1
        if rng.random() < 0.3:
            opts.update(warp_chunks_below=1 << 30, warp_chunk_words=-1)
        if rng.random() < 0.25:
            opts["strict_phase2"] = True
        grid = rng.random() < 0.4
        step, n_scales = int(rng.integers(5000, 60000)), int(rng.integers(1, 8))
        mp = -1 if rng.random() < 0.6 else int(rng.integers(0, 4))
        okw = {"strict": opts.get("strict_phase2", False)}
        if mp >= 0:
            okw["max_passes"] = mp
        x = np.concatenate(clouds)
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        ctx = ph.Context(collect_stats=True, **opts)
        if grid:
            ctx.build_filtration_scales(torch.from_numpy(x).cuda(), off, k, step, n_scales)
        else:
            ctx.build_filtration(torch.from_numpy(x).cuda(), off, k)
        ctx.reduce(max_passes=mp)
        for c, xc in enumerate(clouds):
            K = (orc.vr_build(xc, k, scale_step=step, n_scales=n_scales) if grid
                 else orc.vr_build(xc, k))
            ref = orc.reduce_pms(K, **okw)
            where = (case, c, sizes, D, k, grid, mp, opts)
            f = ctx.filtration(c)
            assert np.array_equal(f["dim"], K["dim"]) and np.array_equal(f["low"], ref.low), where
            cp, rows = orc.reduce_pms_columns(K, **okw)
            gcp, grows = ctx.columns(c)
            assert np.array_equal(gcp, cp) and np.array_equal(grows, rows), where
            # a cloud that converged earlier than the batch is final: later passes leave it be
            assert np.array_equal(ctx.essential_estimate(c), ref.ess_est), where
            if opts["predict_pairs"]:
                assert np.array_equal(ctx.predicted_lows(c), ref.predicted), where
        ctx.close()


_DEBUG_RUN = r"""
import numpy as np, torch
import oracle, pointclouds as pc, paper_1708_04710_gb300 as ph
assert ph.native.LIB_PATH.name == "libph_gb300_debug.so"
oracle.build_lib()
cases = [(pc.circle40(), 2, {}), (pc.random_cloud(11, 3, 31), 4, {"dense_threshold": 1}),
         (pc.random_cloud(60, 3, 12), 2, {"arena_words": 1, "warp_chunks_below": 1 << 30,
                                          "warp_chunk_words": -1}),
         (pc.random_cloud(30, 3, 500), 2, {"phase2_sets": 3, "phase2_priority": 1}),
         (pc.torus400()[:120], 2, {"use_graph": False})]
for x, k, opts in cases:
    K = oracle.vr_build(x, k)
    okw = {"sets": opts.get("phase2_sets", 0), "priority": opts.get("phase2_priority", 0)}
    ref = oracle.reduce_pms(K, **okw)
    cp, rows = oracle.reduce_pms_columns(K, **okw)
    ctx = ph.Context(collect_stats=True, **opts)
    ctx.build_filtration(torch.from_numpy(x).cuda(), None, k)
    st = ctx.reduce()
    assert st["passes"] == ref.passes
    assert np.array_equal(ctx.pass_stats()[:, :8], ref.stats[:, :8])
    gcp, grows = ctx.columns(0)
    assert np.array_equal(gcp, cp) and np.array_equal(grows, rows)
print("debug build ok")
"""


def test_debug_build_bounds_checks_pass(ph):
    # The build with device-side bounds checks (every arena, pivot-store, active-list, row and
    # bitmap access of the pass kernels checked; a failure is reported, not trapped) runs the
    # parity cases clean and exact. It runs in its own process, which loads the debug library.
    import os
    import subprocess
    import sys

    from paper_1708_04710_gb300 import build

    build.build(debug=True)
    env = dict(os.environ, PH_GB300_DEBUG="1")
    root = Path(__file__).resolve().parents[1]
    r = subprocess.run([sys.executable, "-c", _DEBUG_RUN], cwd=root, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "debug build ok" in r.stdout, r.stdout + r.stderr


@pytest.mark.parametrize("mp", [0, 2, 5])
def test_checkpoint_and_resume_through_the_reduced_matrix(ph, orc, mp):
    # a partial reduction saved as its reduced matrix R (ph_get_columns), loaded into a new
    # context (ph_load_boundary) and reduced there: the pairs of the original complex; the
    # resumed run itself is the oracle's run on R, pass by pass
    from oracle import Complex

    for x, k in ((pc.circle40(), 2), (pc.random_cloud(12, 3, 801), 3)):
        K = orc.vr_build(x, k)
        ctx = _gpu(ph, x, k)
        ctx.reduce(max_passes=mp)
        cp, rows = ctx.columns(0)
        dims = ctx.filtration(0)["dim"]
        ctx2 = ph.Context(collect_stats=True)
        ctx2.load_boundary(dims, cp, rows)
        st = ctx2.reduce()
        R = Complex(dim=K["dim"], diam2=K["diam2"], verts=K["verts"], colptr=cp, rows=rows)
        ref_r = orc.reduce_pms(R)
        assert st["passes"] == ref_r.passes
        assert np.array_equal(ctx2.pass_stats()[:, :8], ref_r.stats[:, :8])
        low = ctx2.filtration(0)["low"]
        assert np.array_equal(low, orc.reduce_pms(K).low)


def test_cubical_complex(ph, orc):
    # columns of four rows (squares): the same lows, counters and reduced matrix as the oracle
    from oracle import Complex
    from helpers import cubical_grid

    for w, h in ((3, 3), (7, 5)):
        filled = [(x, y) for x in range(w) for y in range(h) if (x + 2 * y) % 5]
        dims, cp0, rows0 = cubical_grid(w, h, filled)
        K = Complex(dim=dims, diam2=np.zeros(len(dims), np.int64),
                    verts=np.full((len(dims), 4), -1, np.int32), colptr=cp0, rows=rows0)
        ref = orc.reduce_pms(K)
        for opts in ({}, {"dense_threshold": 1, "use_graph": False}):
            ctx = ph.Context(collect_stats=True, **opts)
            ctx.load_boundary(dims, cp0, rows0)
            st = ctx.reduce()
            assert st["passes"] == ref.passes
            assert np.array_equal(ctx.filtration(0)["low"], ref.low)
            assert np.array_equal(ctx.pass_stats()[:, :8], ref.stats[:, :8])
            cp, rows = orc.reduce_pms_columns(K)
            gcp, grows = ctx.columns(0)
            assert np.array_equal(gcp, cp) and np.array_equal(grows, rows)


def _addition_cases(seed=5):
    """A matrix of 4096 rows (dimension 0) and columns built so that the first pass adds, per
    group, a source column into targets with the same low: equal columns, length-1 columns,
    disjoint and nested ones, columns longer than the staging bound, very uneven lengths, and
    one source shared by many targets. Rows of a group lie below its own low."""
    rng = np.random.default_rng(seed)
    n_rows = 4096
    cols = []
    lows = iter(range(n_rows - 1, 0, -7))

    def rand_rows(low, k):
        return np.sort(rng.choice(low, size=min(k, low), replace=False)).tolist() + [low]

    groups = []
    low = next(lows); s = rand_rows(low, 6); groups.append((s, [list(s)]))           # equal
    low = next(lows); groups.append(([low], [[low]]))                                  # length 1
    low = next(lows)
    a = rand_rows(low, 5); b = sorted(set(rand_rows(low, 5)) - set(a[:-1]))
    groups.append((a, [b]))                                                            # disjoint
    low = next(lows); s = rand_rows(low, 40)
    groups.append((s, [sorted(set(s) | set(rand_rows(low, 30)))]))                    # nested
    low = next(lows); groups.append((rand_rows(low, 60), [rand_rows(low, 70)]))       # staged
    low = next(lows); groups.append((rand_rows(low, 900), [rand_rows(low, 1100)]))    # > staging
    low = next(lows); groups.append((rand_rows(low, 2), [rand_rows(low, 1500)]))      # uneven
    low = next(lows); groups.append((rand_rows(low, 1500), [rand_rows(low, 2)]))
    low = next(lows); groups.append((rand_rows(low, 20), [rand_rows(low, int(rng.integers(1, 90)))
                                                         for _ in range(40)]))        # 40 targets
    for src, tgts in groups:
        cols.append(src)
        cols.extend(tgts)
    # every source first (left-most for its low), then the targets in a random order
    order = rng.permutation(len(cols))
    src_idx = set(np.cumsum([0] + [1 + len(t) for _, t in groups[:-1]]).tolist())
    firsts = [c for i, c in enumerate(cols) if i in src_idx]
    rest = [cols[i] for i in order if i not in src_idx]
    cols = firsts + rest
    dims = np.array([0] * n_rows + [1] * len(cols), np.int32)
    lengths = np.cumsum([len(c) for c in cols])
    colptr = np.concatenate([[0] * (n_rows + 1), lengths]).astype(np.int64)
    rows = np.array([r for c in cols for r in c], np.int32)
    return dims, colptr, rows


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("arena_words", [0, 1])
def test_many_passes_counter_rows_and_space_stops(ph, orc, use_graph, arena_words):
    # 299 passes: more than the first 256 rows of per-pass counters, which are grown between
    # two passes; with one-word arenas, passes also stop after their marks for space and continue
    # at Phase II. Lows, pass count and every pass's counters against the oracle.
    from helpers import staircase
    from oracle import Complex

    dims, cp, rows = staircase(300)
    m = len(dims)
    K = Complex(dim=dims, diam2=np.zeros(m, np.int64), verts=np.full((m, 4), -1, np.int32),
                colptr=cp, rows=rows)
    ref = orc.reduce_pms(K)
    assert ref.passes > 256
    ctx = ph.Context(collect_stats=True, use_graph=use_graph, arena_words=arena_words)
    ctx.load_boundary(dims, cp, rows)
    st = ctx.reduce()
    assert st["converged"] and st["passes"] == ref.passes
    assert np.array_equal(ctx.filtration(0)["low"], ref.low)
    assert np.array_equal(ctx.pass_stats()[:, :8], ref.stats[:, :8])


@pytest.mark.parametrize("opts", [{}, {"staged_merge_max": 1}, {"staged_merge_max": 16},
                                  {"dense_threshold": 1},
                                  {"warp_chunks_below": 1 << 30, "warp_chunk_words": -1},
                                  {"use_graph": False, "merge_items": 3},
                                  {"lane_merge_words": -1},
                                  {"lane_merge_words": 1 << 30},
                                  {"lane_merge_words": -1, "warp_chunks_below": 1 << 30,
                                   "warp_chunk_words": -1, "narrow_chunks_below": -1},
                                  {"lane_merge_words": -1, "warp_chunks_below": 1 << 30,
                                   "warp_chunk_words": -1, "narrow_chunks_below": 1 << 30}],
                         ids=["default", "global", "staged16", "bitmaps", "warp", "host_km3",
                              "pieces", "lanes", "pieces_warp32", "pieces_warp8"])
def test_column_additions_edge_cases(ph, orc, opts):
    # the symmetric difference itself on crafted columns, through every merge path: the
    # reduced matrix, lows and counters against the oracle's sorted-array additions
    from oracle import Complex

    dims, cp0, rows0 = _addition_cases()
    K = Complex(dim=dims, diam2=np.zeros(len(dims), np.int64),
                verts=np.full((len(dims), 4), -1, np.int32), colptr=cp0, rows=rows0)
    ref = orc.reduce_pms(K)
    cp, rows = orc.reduce_pms_columns(K)
    ctx = ph.Context(collect_stats=True, **opts)
    ctx.load_boundary(dims, cp0, rows0)
    st = ctx.reduce()
    assert st["passes"] == ref.passes
    assert np.array_equal(ctx.filtration(0)["low"], ref.low)
    assert np.array_equal(ctx.pass_stats()[:, :8], ref.stats[:, :8])
    gcp, grows = ctx.columns(0)
    assert np.array_equal(gcp, cp) and np.array_equal(grows, rows)


@pytest.mark.parametrize("world", [2, 3, 5])
def test_sharded_batch_equals_unsharded(ph, world):
    # the multi-GPU form of the batch shards clouds across ranks with no collective; here the
    # shards run one after another on one GPU, and every cloud's pairs, essentials and
    # reduced matrix equal those of the whole batch reduced together
    import torch

    from paper_1708_04710_gb300.shard import local_batch, shard_clouds

    sizes = [int(s) for s in np.random.default_rng(31).integers(3, 40, 23)]
    clouds = [pc.random_cloud(n, 3, 3000 + i) for i, n in enumerate(sizes)]
    x = np.concatenate(clouds)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    whole = _gpu(ph, x, 2, offsets=off)
    whole.reduce()
    seen = []
    for part in shard_clouds(off, world):
        if not part:
            continue
        xs, offs = local_batch(x, off, part)
        ctx = ph.Context()
        ctx.build_filtration(torch.from_numpy(xs).cuda(), offs, 2)
        assert ctx.reduce()["converged"]
        for i, c in enumerate(part):
            a, b = _gpu_pairs(ctx, i), _gpu_pairs(whole, c)
            for k in ("birth", "death", "dim"):
                assert np.array_equal(a[0][k], b[0][k]), (world, c, k)
            assert np.array_equal(a[1]["idx"], b[1]["idx"]), (world, c)
            ca, cb = ctx.columns(i), whole.columns(c)
            assert np.array_equal(ca[0], cb[0]) and np.array_equal(ca[1], cb[1]), (world, c)
            seen.append(c)
    assert sorted(seen) == list(range(len(sizes)))
