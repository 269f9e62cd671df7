#!/usr/bin/env python
"""Throughput of the persistent-homology hot path: simplices reduced per second to full pairing.

One step = the whole path on one synthetic workload: Vietoris-Rips filtration built on the
device, Algorithm 2 reduction to full pairing, pairs and essential simplices extracted on the
device. The default workload is the complete VR complex up to dimension 2 of 400 seeded points
on the torus (R=2, r=1) in R^3 on the 2^-16 grid: 10,667,000 simplices.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (VR build + Algorithm 3, one core) on a bounded sample of
the same workload. Under torchrun every rank reduces its own replica of the workload (a single
filtration does not shard); value is the total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

import pointclouds as pc  # noqa: E402

METRIC = "simplices reduced/sec to full pairing (bit-exact vs oracle), passes, % HBM roofline"
UNIT = "simplices/s"
PEAKS = ROOT / "MEASURED_PEAKS.json"
FALLBACK_HBM = 6800.0

WORKLOADS = {
    "torus400": dict(gen=pc.torus400, max_dim=2, max_diam2=-1,
                     desc="complete VR <= dim 2, 400 points on the torus R=2 r=1 in R^3"),
    "circle40": dict(gen=pc.circle40, max_dim=2, max_diam2=-1,
                     desc="complete VR <= dim 2, 40 noisy points on the unit circle"),
    "gauss8_120": dict(gen=pc.gauss8_120, max_dim=3, max_diam2=pc.GAUSS8_MAX_DIAM2,
                       desc="VR <= dim 3, 120 points N(0, I_8), squared diameter <= 16"),
    # smaller case of the same law for ncu captures (2.6M simplices)
    "torus250": dict(gen=lambda: pc.torus400()[:250], max_dim=2, max_diam2=-1,
                     desc="complete VR <= dim 2, first 250 of the 400 torus points"),
    # the batched form: independent clouds, sharded across ranks under torchrun
    "batch512": dict(gen=pc.batch512, max_dim=2, max_diam2=-1, batched=True,
                     desc="512 clouds, n ~ U{20..120}, sphere/torus/N(0,I3), complete VR <= dim 2"),
}


def _peak_hbm():
    try:
        return float(json.loads(PEAKS.read_text())["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def _profile_traffic(kernel: str, workload: str):
    """dram bytes per launch of `kernel` recorded by the committed ncu summary, if any."""
    p = ROOT / "profiles" / f"{kernel}_{workload}.md"
    if not p.exists():
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", p.read_text())
    return float(m.group(1)) if m else None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        with open(self.f.name) as f:
            lines = f.readlines()
        os.unlink(self.f.name)
        return parse_clocks(lines)


def parse_clocks(lines):
    """Median SM clock, maximum clock and the throttle reasons seen in nvidia-smi samples
    (index, clocks.sm, clocks.max.sm, power.draw, active mask, then the four reasons)."""
    rows = []
    for line in lines:
        parts = [s.strip() for s in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v == "Active"})
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_oracle_sample(n_sample: int):
    """The oracle as it stands (VR build + Algorithm 3) on the first n_sample points of the
    torus workload; returns (simplices, seconds)."""
    import oracle

    oracle.build_lib()
    x = pc.torus400()[:n_sample]
    t0 = time.perf_counter()
    K = oracle.vr_build(x, 2)
    oracle.reduce_twist(K)
    return K.m, time.perf_counter() - t0


def run_reference(args, rank):
    if rank != 0:
        return
    n_sample = 200
    for _ in range(args.warmup):
        cpu_oracle_sample(n_sample)
    times, m = [], 0
    for _ in range(args.steps):
        m, t = cpu_oracle_sample(n_sample)
        times.append(t)
    total = sum(times)
    value = m * len(times) / total
    sample = (f"first {n_sample} of the 400 torus points: complete VR <= dim 2, m={m}; "
              "oracle VR build + Algorithm 3 (twist), one core, per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "sample_points": n_sample, "m": m},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="torus400", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="library default options (short profiler captures)")
    ap.add_argument("--pass-loop", default="graph", choices=["graph", "host"],
                    help="pass loop of the timed steps: one CUDA graph, or host-driven")
    ap.add_argument("--experiment", choices=["early"],
                    help="instead of the throughput line: early-stopping quality per iteration "
                         "on the four 15-point ensembles (complete complex to dimension 5)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.experiment == "early":
        return run_early()

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1708_04710_gb300 import build as _build

    _build.build()
    import paper_1708_04710_gb300 as ph

    wl = WORKLOADS[args.workload]
    offsets = None
    if wl.get("batched"):
        from paper_1708_04710_gb300.shard import local_batch, shard_clouds

        xa, off_all = wl["gen"]()
        mine = shard_clouds(off_all, world)[rank]  # independent clouds: no collective needed
        x, offsets = local_batch(xa, off_all, mine)
    else:
        x = wl["gen"]()  # one filtration does not shard: every rank reduces a replica
    coords = torch.from_numpy(x).to(dev)
    from paper_1708_04710_gb300 import autotune

    tuned = ({} if args.no_autotune
             else autotune.tune(coords, offsets, wl["max_dim"], wl["max_diam2"]))
    # the pass loop runs in one CUDA graph by default
    ctx = ph.Context(**dict(tuned, use_graph=args.pass_loop == "graph"))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step(c, context=ctx, marks=None):
        context.build_filtration(c, offsets, wl["max_dim"], wl["max_diam2"])
        if marks:
            marks[0].record(stream)
        st = context.reduce()
        if marks:
            marks[1].record(stream)
        context.pairs(-1, on_device=True)
        context.essential(-1, on_device=True)
        return st

    for _ in range(max(args.warmup, 0)):
        step(coords)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(dev.index) if rank == 0 else None
    launches0 = ctx.kernel_launches()
    total_ms, stats = 0.0, []
    phase_ms = [0.0, 0.0, 0.0]  # filtration build, reduction, extraction
    for _ in range(args.steps):
        flush.fill_(1)  # write 256 MiB (> 129 MB L2) so no step starts from a warm L2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e0.record(stream)
        stats.append(step(coords, marks=marks))
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        phase_ms[0] += e0.elapsed_time(marks[0])
        phase_ms[1] += marks[0].elapsed_time(marks[1])
        phase_ms[2] += marks[1].elapsed_time(e1)
    torch.cuda.synchronize()
    launches = ctx.kernel_launches() - launches0
    clk = clocks.stop() if clocks else None
    t_max = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if dist:
        dist.barrier()
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    total_ms = float(t_max.item())
    m_local = ctx.m
    m_all = torch.tensor([float(m_local)], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(m_all, op=dist.ReduceOp.SUM)
    m = int(m_all.item())  # simplices reduced per step by all ranks together
    value = m * args.steps / (total_ms / 1000.0)

    # end to end through the public API with host buffers: H2D of the coordinates and D2H of
    # every output (pairs and essential simplices) inside the timed region
    x_pin = torch.from_numpy(x).pin_memory()
    dev_buf = torch.empty_like(coords)
    e2e_times, d2h = [], 0
    # two untimed steps first: the page-locked output buffers (two generations, since a step's
    # outputs are still alive when the next is requested) come from torch's host cache after
    for it in range(2 + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dev_buf.copy_(x_pin, non_blocking=True)
        ctx.build_filtration(dev_buf, offsets, wl["max_dim"], wl["max_diam2"])
        ctx.reduce()
        pr = ctx.pairs(-1, on_device=False)
        es = ctx.essential(-1, on_device=False)
        torch.cuda.synchronize()
        if it >= 2:
            e2e_times.append(time.perf_counter() - t0)
        d2h = sum(v.numel() * v.element_size() for v in list(pr.values()) + list(es.values()))
    e2e_s = torch.tensor([sum(e2e_times)], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(e2e_s, op=dist.ReduceOp.MAX)
    e2e_value = m * args.steps / float(e2e_s.item())

    # parity of the last output against the stored oracle result
    parity = None
    gpath = ROOT / "tests" / "golden" / f"{args.workload}.json"
    if gpath.exists() and not wl.get("batched"):
        g = json.loads(gpath.read_text())
        b, d = pr["birth"].numpy(), pr["death"].numpy()
        o = np.lexsort((b, d))
        p = np.stack([b[o], d[o]], 1).astype(np.int64)
        e = np.sort(es["idx"].numpy()).astype(np.int64)
        parity = (hashlib.sha256(p.tobytes()).hexdigest() == g["pairs_sha"]
                  and hashlib.sha256(e.tobytes()).hexdigest() == g["ess_sha"]
                  and stats[-1]["passes"] == g["passes"])

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # the dominant kernel, k_add, timed with CUDA events on the library's stream around every
    # launch: the same workload through the host-driven pass loop (events cannot sit inside the
    # graph's conditional body), with per-pass counters for its algorithmic bytes
    prof = ph.Context(**dict(tuned, use_graph=False, collect_stats=True, time_kernels=True))
    step(coords, prof)
    peak, peak_kind = _peak_hbm()
    roofline = kadd_roofline(ph, prof, lambda: step(coords, prof), peak, peak_kind)
    roofline["traffic"] = _profile_traffic("k_add", args.workload)
    roofline["share_of_step"] = roofline.pop("_ms_per_reduction") / (total_ms / args.steps)
    # the same reduction through the timed graph loop and through the host-driven loop (whose
    # k_add launches the events above time), each reduction alone, after a warm-up
    roofline["reduce_ms_graph_loop"] = _reduce_ms(torch, ph, tuned, coords, offsets, wl, True)
    roofline["reduce_ms_host_loop"] = _reduce_ms(torch, ph, tuned, coords, offsets, wl, False)
    pst = [roofline.pop("_last_stats")]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "m": m,
                       "parallelism": (f"clouds sharded x{world}" if wl.get("batched") else
                                       f"replicas x{world}") if world > 1 else "single",
                       "pass_loop": ("CUDA graph, conditional while node"
                                     if args.pass_loop == "graph" else "host-driven"),
                       "autotuned": tuned,
                       "l2": "256 MiB buffer written before every timed step"},
            "passes": stats[-1]["passes"], "col_adds": pst[-1]["col_adds"],
            "xors": pst[-1]["xors"], "bit_exact_vs_oracle": parity,
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(x.nbytes),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches), "clocks": clk,
            # the step's three parts, same timed steps (rank 0's clock)
            "phases": {name: {"ms": t / args.steps,
                              "simplices_per_s": m_local * args.steps / (t / 1e3) if t else None}
                       for name, t in zip(("build_filtration", "reduce", "extract"), phase_ms)}}
    # the build against the bytes a filtration must write: 16 B per simplex (diameter and
    # vertex tuple), 4 B per boundary nonzero, 4 B of beta per simplex
    counts = np.bincount(ctx.filtration(0)["dim"], minlength=1) if not wl.get("batched") else None
    if counts is not None and phase_ms[0]:
        nnz = int(sum((d + 1) * int(c) for d, c in enumerate(counts) if d > 0))
        b_bytes = 20 * m_local + 4 * nnz
        b_gbs = b_bytes / (phase_ms[0] / args.steps / 1e3) / 1e9
        line["phases"]["build_filtration"]["roofline"] = {
            "bound": "hbm", "achieved": b_gbs, "peak": peak, "unit": "GB/s", "frac": b_gbs / peak,
            "bytes": b_bytes, "nnz": nnz}
    if world == 1 and not args.no_forms and not wl.get("batched"):
        line["forms"] = compare_forms(ph, torch, dev)
        line["configs"] = other_configs(ph, torch, dev, peak, peak_kind)
        line["early"] = early_summary(ph, torch)
        line["packed"] = packed_summary(ph, torch, dev)
    if world == 1 and not args.no_cpu_baseline:
        n_sample = 250
        ms, secs = cpu_oracle_sample(n_sample)
        live = {"value": ms / secs, "unit": UNIT, "cores": 1,
                "sample": f"first {n_sample} of the 400 torus points: complete VR <= dim 2, "
                          f"m={ms}; oracle VR build + Algorithm 3 (twist), {secs:.1f} s on one "
                          "core of this host, timed in this run"}
        host, cached = cached_oracle_times()
        full = (cached or {}).get("workloads", {}).get(args.workload)
        if full:
            line["cpu_baseline"] = {
                "value": full["simplices_per_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"the whole {args.workload} workload (m={full['m']}): oracle VR build "
                          f"({full['build_s']} s) + Algorithm 3 (twist, {full['reduce_s']} s) "
                          f"on one core of a GB300 box's host ({cached['cpu']}, {host}), timed "
                          "once by tests/golden/time_oracle.py and stored",
                "reduce_only_simplices_per_s": full["reduce_simplices_per_s"],
                "live_subsample": live}
        else:
            line["cpu_baseline"] = dict(live, kind="oracle")
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# algorithmic bytes of the additions kernel, per the method's minimum traffic: 8 B per nontrivial
# XOR (4 * (|src| + |tgt| + |out|) = 8 * |src union tgt|) and 26 B per active column per pass
# (column header and low read 4, low write 4, table atomic 4, table read 4, flags 1, active list
# read and write 8 -- charged to k_add, which dominates the pass)
BYTES_PER_XOR = 8
BYTES_PER_ACTIVE = 26


def kadd_roofline(ph, prof, run_step, peak, peak_kind, reps=2):
    """k_add's achieved algorithmic bandwidth: CUDA events around every k_add launch of `reps`
    host-driven reductions (library stream), bytes from the same reductions' per-pass counters
    (active columns and XORs; the rows copied without an addition are reported apart)."""
    xors = active = copied = launches = 0
    ms = 0.0
    st = None
    for _ in range(reps):
        st = run_step()
        ps = prof.pass_stats()
        xors += int(ps[:, ph.PS_FIELDS.index("xors")].sum())
        active += int(ps[:, ph.PS_FIELDS.index("active")].sum())
        copied += int(ps[:, ph.PS_FIELDS.index("copied")].sum())
        launches += st["add_launches"]
        ms += st["ms_add"]
    nbytes = BYTES_PER_XOR * xors + BYTES_PER_ACTIVE * active
    per_launch_ms = ms / max(launches, 1)
    achieved = nbytes / max(launches, 1) / (per_launch_ms / 1e3) / 1e9 if ms else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": None,
            "kernel": "k_add (Phase II column additions)", "peak_kind": peak_kind,
            "bytes_per_launch": nbytes / max(launches, 1),
            "bytes_model": f"{BYTES_PER_XOR} B per nontrivial XOR + {BYTES_PER_ACTIVE} B per "
                           "active column per pass (counters below, per reduction)",
            "xors_per_reduction": xors // reps, "active_column_passes_per_reduction": active // reps,
            "copied_rows_per_reduction": copied // reps,
            "copied_row_bytes_per_launch": 8 * copied / max(launches, 1),
            "ms_per_launch": per_launch_ms, "launches_per_step": launches / reps,
            "timing": f"CUDA events around each k_add launch, host-driven pass loop, same "
                      f"workload, {reps} reductions after 1 warm-up",
            "_ms_per_reduction": ms / reps, "_last_stats": st}


def _reduce_ms(torch, ph, tuned, coords, offsets, wl, graph, reps=3):
    """Median CUDA-event time of ph_reduce alone on a freshly built filtration."""
    ctx = ph.Context(**dict(tuned, use_graph=graph))
    stream = torch.cuda.current_stream()
    times = []
    for it in range(reps + 1):
        ctx.build_filtration(coords, offsets, wl["max_dim"], wl["max_diam2"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.reduce()
        e1.record(stream)
        e1.synchronize()
        if it:
            times.append(e0.elapsed_time(e1))
    ctx.close()
    return statistics.median(times)


def _golden(name):
    p = ROOT / "tests" / "golden" / f"{name}.json"
    return json.loads(p.read_text()) if p.exists() else None


def _canon_sha(pr, es):
    """SHA-256 of the canonical pairs (sorted by death, then birth) and essential indices."""
    b, d = pr["birth"].cpu().numpy(), pr["death"].cpu().numpy()
    o = np.lexsort((b, d))
    p = np.stack([b[o], d[o]], 1).astype(np.int64)
    e = np.sort(es["idx"].cpu().numpy()).astype(np.int64)
    return (hashlib.sha256(p.tobytes()).hexdigest(), hashlib.sha256(e.tobytes()).hexdigest(),
            p, e)


def other_configs(ph, torch, dev, peak, peak_kind):
    """The single-filtration configurations besides the headline one (circle40, gauss8_120):
    the same step (build + reduce + extract, CUDA events, L2 flushed before each), passes,
    bit-exactness against the oracle's stored result, and k_add's roofline fraction."""
    from paper_1708_04710_gb300 import autotune

    out = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    for name in ("circle40", "gauss8_120"):
        wl = WORKLOADS[name]
        coords = torch.from_numpy(wl["gen"]()).to(dev)
        tuned = autotune.tune(coords, None, wl["max_dim"], wl["max_diam2"])
        ctx = ph.Context(**tuned)
        times = []
        for it in range(3 + 10):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.build_filtration(coords, None, wl["max_dim"], wl["max_diam2"])
            st = ctx.reduce()
            pr = ctx.pairs(0, on_device=True)
            es = ctx.essential(0, on_device=True)
            e1.record(stream)
            e1.synchronize()
            if it >= 3:
                times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        g = _golden(name)
        ps, es_sha, _, _ = _canon_sha(pr, es)
        exact = (g is not None and ps == g["pairs_sha"] and es_sha == g["ess_sha"]
                 and st["passes"] == g["passes"])
        prof = ph.Context(**dict(tuned, use_graph=False, collect_stats=True, time_kernels=True))

        def run(prof=prof, coords=coords, wl=wl):
            prof.build_filtration(coords, None, wl["max_dim"], wl["max_diam2"])
            return prof.reduce()

        run()
        rl = kadd_roofline(ph, prof, run, peak, peak_kind)
        rl.pop("_last_stats")
        rl.pop("_ms_per_reduction")
        out[name] = {"desc": wl["desc"], "m": ctx.m, "ms_per_step": ms,
                     "simplices_per_s": ctx.m / (ms / 1e3), "passes": st["passes"],
                     "bit_exact_vs_oracle": exact, "autotuned": tuned,
                     "k_add": {k: rl[k] for k in ("achieved", "frac", "bytes_per_launch",
                                                   "ms_per_launch", "launches_per_step")}}
        ctx.close()
        prof.close()
    return out


def packed_summary(ph, torch, dev):
    """The bit-packed column path, timed on two small complexes: 24 random points to dimension 4
    (55,454 simplices) and circle40 (10,700), each reduced with row lists only (dense_threshold
    -1), the default threshold (0: a column goes bit-packed once its bitmap is the smaller form,
    past 32 rows) and every addition past one row bit-packed (1). Per variant: the reduction's
    median time (graph loop, 10 runs after 3 warm-ups), passes, and the additions computed on
    bitmaps; the variants of a complex must agree on every low."""
    out = {}
    for name, x, k in (("rand24_dim4", pc.random_cloud(24, 3, 77), 4), ("circle40", pc.circle40(), 2)):
        coords = torch.from_numpy(x).to(dev)
        res = {"variants": {}}
        lows = []
        for var, thr in (("row_lists", -1), ("default", 0), ("forced", 1)):
            ctx = ph.Context(dense_threshold=thr)
            times = []
            for it in range(3 + 10):
                ctx.build_filtration(coords, None, k)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                st = ctx.reduce()
                e1.record()
                e1.synchronize()
                if it >= 3:
                    times.append(e0.elapsed_time(e1))
            cnt = ph.Context(dense_threshold=thr, collect_stats=True)
            cnt.build_filtration(coords, None, k)
            cnt.reduce()
            ps = cnt.pass_stats()
            lows.append(cnt.filtration(0)["low"])
            res["m"] = ctx.m
            res["variants"][var] = {
                "dense_threshold": thr, "reduce_ms": statistics.median(times),
                "passes": st["passes"],
                "packed_additions": int(ps[:, ph.PS_FIELDS.index("packed")].sum()),
                "additions": int(ps[:, ph.PS_FIELDS.index("adds")].sum())}
            ctx.close()
            cnt.close()
        res["same_lows"] = all(np.array_equal(lows[0], lw) for lw in lows[1:])
        out[name] = res
    return out


def early_summary(ph, torch):
    """Early stopping on the four 15-point stand-in ensembles (complete VR to dimension 5 on the
    paper's scale grid): passes, additions, and the iterations Algorithm 2 needs to reach an
    l1 error of 0.01 and an essential-estimate precision of 0.95 and 1.0 (Sec. 4.2-4.3), for
    the default rule and for the paper's rule without Corollary 10's zero case."""
    from paper_1708_04710_gb300 import early

    step, n_scales = pc.GRID_SCALE // 2, 10
    res = {}
    for name in pc.ENSEMBLES:
        x = torch.from_numpy(pc.ensemble15(name)).cuda()
        res[name] = {}
        for mode, strict, cor10 in (("default", False, True), ("paper_rule", True, False)):
            ctx = ph.Context(collect_stats=True, strict_phase2=strict, use_cor10=cor10)
            ctx.build_filtration_scales(x, None, 5, step, n_scales)
            pr = early.profile(ctx)
            res[name][mode] = {
                "m": pr["m"], "passes": pr["passes"], "adds": pr["adds"][-1],
                "to_l1_0.01": early.iterations_to(pr["l1_error"], [0.01])[0.01],
                "to_precision_0.95": early.iterations_to(pr["precision"], [0.95],
                                                         below=False)[0.95],
                "to_precision_1.0": early.iterations_to(pr["precision"], [1.0],
                                                        below=False)[1.0]}
            ctx.close()
    return res


def cached_oracle_times():
    """The oracle's full-size times stored by tests/golden/time_oracle.py (GPU machine host first)."""
    p = ROOT / "tests" / "golden" / "oracle_times.json"
    if not p.exists():
        return None, None
    data = json.loads(p.read_text())
    for key in ("aarch64", "x86_64"):
        if key in data:
            return key, data[key]
    return None, None


def run_early():
    """Iterations of Algorithm 2 to given levels of relative l1 error of low (Eq. rel_error),
    unreduced share and essential-estimate precision, per ensemble, for the left-most source
    (default), the printed rule (strict_phase2), and Phase II limited to 32 neighbour sets per
    pass under both orders of Sec. 3.4. One JSON line."""
    import torch

    from paper_1708_04710_gb300 import build as _build

    _build.build()
    import paper_1708_04710_gb300 as ph
    from paper_1708_04710_gb300 import early

    torch.cuda.set_device(0)
    step, n_scales = pc.GRID_SCALE // 2, 10  # the paper's grid: r_T = 5 in h = 10 divisions
    res = {}
    for name in pc.ENSEMBLES:
        x = torch.from_numpy(pc.ensemble15(name)).cuda()
        res[name] = {}
        # the last two: p = 32 processors, the sets of Sec. 3.4.1 (largest first) against
        # those of Sec. 3.4.2 (known-negative targets first)
        for mode, strict, cor10, sets, prio in (
                ("leftmost", False, True, 0, 0), ("strict", True, True, 0, 0),
                ("leftmost_no_cor10", False, False, 0, 0), ("strict_no_cor10", True, False, 0, 0),
                ("p32_largest_sets_first", False, False, 32, 0),
                ("p32_negatives_first", False, False, 32, 1)):
            ctx = ph.Context(collect_stats=True, strict_phase2=strict, use_cor10=cor10,
                             phase2_sets=sets, phase2_priority=prio)
            ctx.build_filtration_scales(x, None, 5, step, n_scales)
            pr = early.profile(ctx)
            res[name][mode] = {
                "m": pr["m"], "passes": pr["passes"], "ess": pr["ess"],
                "total_adds": pr["adds"][-1], "total_xors": pr["xors"][-1],
                "iterations_to_l1_error": early.iterations_to(
                    pr["l1_error"], [0.1, 0.01, 0.001, 0.0001, 0.0]),
                "iterations_to_unreduced": early.iterations_to(
                    pr["unreduced"], [0.9, 0.5, 0.1, 0.05, 0.01]),
                "iterations_to_precision": early.iterations_to(
                    pr["precision"], [0.1, 0.5, 0.9, 0.95, 1.0], below=False),
                "precision": [round(v, 4) for v in pr["precision"]],
            }
    print(json.dumps({"experiment": "early", "data": "synthetic",
                      "desc": "15 points per ensemble, VR complex to dimension 5 on the scale "
                              "grid r_i = 0.5 i, i <= 10",
                      "results": res}), flush=True)


def _timed(torch, fn, reps=2):
    fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps


def compare_forms(ph, torch, dev):
    """The batched and differentiable forms against the plain form on the same GPU."""
    out = {}
    # batched: 512 uneven clouds in one filtration vs one plain filtration per cloud
    xb, off = pc.batch512()
    cb = torch.from_numpy(xb).to(dev)
    ctx = ph.Context()

    def batched():
        ctx.build_filtration(cb, off, 2)
        ctx.reduce()
        ctx.pairs(0)

    def looped():
        for c in range(len(off) - 1):
            ctx.build_filtration(cb[off[c]:off[c + 1]].contiguous(), None, 2)
            ctx.reduce()
            ctx.pairs(0)

    tb = _timed(torch, batched)
    mb = ctx.m
    # every cloud's pairs and essentials against the oracle's stored digest of all of them
    batched()
    h = hashlib.sha256()
    for c in range(len(off) - 1):
        _, _, p_c, e_c = _canon_sha(ctx.pairs(c, on_device=False),
                                    ctx.essential(c, on_device=False))
        h.update(p_c.tobytes())
        h.update(e_c.tobytes())
    gb = _golden("batch512")
    tl = _timed(torch, looped, reps=1)
    out["batched"] = {"workload": "batch512: 512 clouds, n ~ U{20..120}, sphere/torus/N(0,I3), "
                                  "complete VR <= dim 2", "m": mb,
                      "batched_simplices_per_s": mb / tb, "looped_plain_simplices_per_s": mb / tl,
                      "batched_ms": 1e3 * tb, "looped_plain_ms": 1e3 * tl,
                      "bit_exact_vs_oracle": gb is not None and h.hexdigest() == gb["all_sha"]}
    # differentiable: loss + gradient over 256 clouds vs the plain build + reduce of the same
    from paper_1708_04710_gb300.diff import diagram_loss

    xd, offd = pc.diff256()
    cd = torch.from_numpy(xd).to(dev)
    dctx = ph.Context()

    def fwd_bwd():
        xx = cd.clone().requires_grad_(True)
        diagram_loss(xx, offd, 1, dctx).sum().backward()

    def plain():
        dctx.build_filtration_f32(cd, offd, 2)
        dctx.reduce()

    tf = _timed(torch, fwd_bwd)
    tp = _timed(torch, plain)
    # every cloud's pairing and loss against the oracle's stored values
    gd = _golden("diff256")
    lossd = diagram_loss(cd, offd, 1, dctx).detach().cpu().numpy()
    exact = gd is not None
    loss_rel = 0.0
    for c in range(len(offd) - 1) if gd is not None else ():
        ps, es_sha, _, _ = _canon_sha(dctx.pairs(c, on_device=False),
                                      dctx.essential(c, on_device=False))
        gc = gd["clouds"][c]
        exact &= ps == gc["pairs_sha"] and es_sha == gc["ess_sha"]
        loss_rel = max(loss_rel, abs(float(lossd[c]) - gc["loss"]) / gc["loss"])
    out["differentiable"] = {"workload": "diff256: 256 clouds x 64 points on S^2 + noise, "
                                         "complete VR <= dim 2, loss over H1 pairs",
                             "m": dctx.m, "forward_backward_ms": 1e3 * tf,
                             "plain_build_reduce_ms": 1e3 * tp,
                             "forward_backward_simplices_per_s": dctx.m / tf,
                             "plain_simplices_per_s": dctx.m / tp,
                             "bit_exact_vs_oracle": bool(exact),
                             "max_loss_rel_err_vs_oracle_fp64": loss_rel}
    return out


if __name__ == "__main__":
    main()
