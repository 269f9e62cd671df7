"""Host-side logic that needs no GPU: the autotuner's search, cache key and cache file, the
sharding of the batched form, the multi-rank aggregation of bench timings over gloo (world size
2), and the bench's roofline arithmetic and clock-sample parsing."""
import os

import numpy as np
import pytest

import pointclouds as pc


def test_coordinate_descent_finds_separable_optimum():
    from paper_1708_04710_gb300.autotune import DEFAULTS, KNOBS, coordinate_descent

    target = {"staged_merge_max": 512, "add_blocks_per_sm": 3, "dense_threshold": -1,
              "warp_chunks_below": 1 << 20, "lane_merge_words": 16, "narrow_chunks_below": -1}

    def timer(o):  # separable cost with its minimum at `target`
        return 1.0 + sum(abs(KNOBS[k].index(o[k]) - KNOBS[k].index(target[k])) for k in KNOBS)

    best, t, trials = coordinate_descent(timer, KNOBS, DEFAULTS)
    assert best == target and t == 1.0
    assert len(trials) == 1 + sum(len(v) - 1 for v in KNOBS.values())


def test_autotune_cache_keeps_other_entries(tmp_path):
    from paper_1708_04710_gb300.autotune import load_cache, store_entry

    path = tmp_path / "sub" / "autotune.json"
    assert load_cache(path) == {}
    store_entry(path, "a", {"options": {"x": 1}})
    store_entry(path, "b", {"options": {"x": 2}})  # as another process would, after "a"
    assert load_cache(path) == {"a": {"options": {"x": 1}}, "b": {"options": {"x": 2}}}
    path.write_text("{ half a fil")  # unreadable: treated as empty, then replaced whole
    assert load_cache(path) == {}
    store_entry(path, "c", {"options": {}})
    assert load_cache(path) == {"c": {"options": {}}}
    assert [p.name for p in path.parent.iterdir()] == ["autotune.json"]


def test_workload_key_classes():
    from paper_1708_04710_gb300.autotune import workload_key

    assert workload_key("GB300", 10_667_000, 2, 1) == workload_key("GB300", 11_000_000, 2, 1)
    assert workload_key("GB300", 10_667_000, 2, 1) != workload_key("GB300", 10_667_000, 2, 512)
    assert workload_key("GB300", 10_667_000, 2, 1) != workload_key("GB300", 1_100_000, 3, 1)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_clouds_partition_and_balance(world):
    from paper_1708_04710_gb300.shard import estimated_work, shard_clouds

    _, off = pc.batch512()
    parts = shard_clouds(off, world)
    flat = sorted(c for p in parts for c in p)
    assert flat == list(range(len(off) - 1))  # disjoint, complete
    w = estimated_work(off)
    loads = [w[p].sum() for p in parts]
    assert max(loads) <= sum(loads) / world + w.max()  # LPT bound


def test_local_batch_roundtrip():
    from paper_1708_04710_gb300.shard import local_batch

    x, off = pc.batch512(n_clouds=7)
    xs, offs = local_batch(x, off, [5, 1, 3])
    assert np.array_equal(xs[offs[0]:offs[1]], x[off[5]:off[6]])
    assert np.array_equal(xs[offs[2]:offs[3]], x[off[3]:off[4]])


def _gloo_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1708_04710_gb300.shard import shard_clouds

    _, off = pc.batch512(n_clouds=64)
    mine = shard_clouds(off, world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)
    # the bench's aggregation: slowest rank's time, total work over ranks
    t = torch.tensor([10.0 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    work = torch.tensor([float(len(mine))], dtype=torch.float64)
    dist.all_reduce(work, op=dist.ReduceOp.SUM)
    q.put((rank, got, float(t.item()), float(work.item())))
    dist.destroy_process_group()


def test_two_rank_sharding_over_gloo():
    import multiprocessing as mp
    import socket

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_gloo_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, g0, t0, w0), (_, g1, t1, w1) = res
    assert g0 == g1  # both ranks agree on the assignment without exchanging data
    assert sorted(g0[0] + g0[1]) == list(range(64)) and not set(g0[0]) & set(g0[1])
    assert t0 == t1 == 11.0 and w0 == w1 == 64.0


def test_kadd_roofline_arithmetic():
    """The bench's k_add figure: 8 B per nontrivial XOR + 26 B per active column per pass,
    over CUDA-event time per launch, against the peak; counters and times from fakes."""
    import bench

    class FakePh:
        PS_FIELDS = ("active", "xors", "copied")

    class FakeProfile:
        def pass_stats(self):
            return np.array([[100, 1000, 5], [50, 500, 0]], np.int64)  # two passes

    rl = bench.kadd_roofline(FakePh, FakeProfile(), lambda: {"add_launches": 4, "ms_add": 2.0},
                             peak=6000.0, peak_kind="measured", reps=2)
    nbytes = 2 * (8 * 1500 + 26 * 150)            # two reductions
    per_launch_s = 2 * 2.0 / 8 / 1e3               # 8 launches in 4 ms
    achieved = nbytes / 8 / per_launch_s / 1e9
    assert rl["achieved"] == pytest.approx(achieved)
    assert rl["frac"] == pytest.approx(achieved / 6000.0)
    assert rl["bytes_per_launch"] == pytest.approx(nbytes / 8)
    assert rl["xors_per_reduction"] == 1500 and rl["active_column_passes_per_reduction"] == 150
    assert rl["copied_row_bytes_per_launch"] == pytest.approx(8 * 10 / 8)  # reported apart
    assert rl["bound"] == "hbm" and rl["unit"] == "GB/s" and rl["traffic"] is None


def test_clock_samples_parsed():
    import bench

    lines = ["0, 2070, 2070, 910.5, 0x0000000000000000, Not Active, Not Active, Not Active, "
             "Not Active\n",
             "0, 1980, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, "
             "Active\n",
             "0, 2040, 2070, 1200.0, 0x0000000000000008, Active, Not Active, Not Active, "
             "Not Active\n",
             "garbled line\n"]
    c = bench.parse_clocks(lines)
    assert c == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "samples": 3,
                 "reasons": ["hw_slowdown", "sw_power_cap"]}
    assert bench.parse_clocks([]) is None
