"""Times the CPU oracle on every full-size workload, one core, and stores the times.

For each workload: the oracle's Vietoris-Rips build and its Algorithm 3 (standard reduction
with clearing), timed separately with a monotonic clock, in one single-threaded process. The
batched and differentiable workloads are timed cloud by cloud and summed (the oracle reduces one
filtration at a time). The results go to oracle_times.json under a key naming the host's
architecture, with the CPU model and core count, so a run on one machine never overwrites
another machine's figures.

    python tests/golden/time_oracle.py [circle40 torus400 gauss8_120 batch512 diff256]

Takes about five minutes on one core (torus400 alone: about two).
"""
from __future__ import annotations

import datetime
import json
import os
import platform
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
import pointclouds as pc  # noqa: E402

OUT = Path(__file__).resolve().parent / "oracle_times.json"


def _cpu_model() -> str:
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except Exception:
        return platform.processor() or "unknown"
    for line in txt.splitlines():
        if line.split(":")[0].strip() in ("Model name", "Model"):
            v = line.split(":", 1)[1].strip()
            if v and not v.isdigit():
                return v
    return platform.processor() or "unknown"


def _one(coords, max_dim, max_diam2=-1):
    t0 = time.perf_counter()
    K = oracle.vr_build(coords, max_dim, max_diam2)
    t1 = time.perf_counter()
    oracle.reduce_twist(K)
    t2 = time.perf_counter()
    return K.m, t1 - t0, t2 - t1


def time_workload(name):
    if name in ("batch512", "diff256"):
        x, off = pc.batch512() if name == "batch512" else pc.diff256()
        m = tb = tr = 0
        for c in range(len(off) - 1):
            xc = x[off[c]:off[c + 1]]
            if name == "diff256":
                xc = pc.to_grid(xc.astype("float64"))
            mc, b, r = _one(xc, 2)
            m, tb, tr = m + mc, tb + b, tr + r
        return m, tb, tr
    if name == "circle40":
        return _one(pc.circle40(), 2)
    if name == "torus400":
        return _one(pc.torus400(), 2)
    if name == "gauss8_120":
        return _one(pc.gauss8_120(), 3, pc.GAUSS8_MAX_DIAM2)
    raise SystemExit(f"unknown workload {name}")


def main(names):
    oracle.build_lib()
    data = json.loads(OUT.read_text()) if OUT.exists() else {}
    key = platform.machine()
    host = data.get(key, {})
    host.update({"cpu": _cpu_model(), "logical_cpus": os.cpu_count(), "cores_used": 1,
                 "when": datetime.datetime.now(datetime.timezone.utc).strftime(
                     "%Y-%m-%dT%H:%M:%SZ")})
    res = host.setdefault("workloads", {})
    for name in names:
        m, tb, tr = time_workload(name)
        res[name] = {"m": int(m), "build_s": round(tb, 3), "reduce_s": round(tr, 3),
                     "total_s": round(tb + tr, 3),
                     "simplices_per_s": round(m / (tb + tr), 1) if tb + tr > 0 else None,
                     "reduce_simplices_per_s": round(m / tr, 1) if tr > 0 else None}
        print(name, res[name], flush=True)
    data[key] = host
    data["generated_by"] = "tests/golden/time_oracle.py (oracle only, one core)"
    OUT.write_text(json.dumps(data, indent=1, sort_keys=True) + "\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["circle40", "gauss8_120", "diff256", "torus400", "batch512"])
