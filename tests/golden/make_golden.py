"""Writes the expected results of the full-size workloads, computed by the CPU oracle only.

For each workload: the SHA-256 of the generated int32 grid coordinates (so a test can tell
generator drift from a kernel bug), the number of simplices per dimension, the persistence pairs
and essential simplices (as SHA-256 of canonical int64 arrays, plus counts per dimension), and
the per-pass counters of the oracle's pass-by-pass Algorithm 2 (default rule: left-most source,
Corollary 10 on). Pairs are checked against Algorithm 3 (twist) before anything is written.
For the differentiable workload (diff256): per cloud, the pairs and essentials as above (from
Algorithm 3 on the grid copy), the fp64 diagram loss over the H1 pairs and the max-abs and l1
norms of its fp64 gradient.

    python tests/golden/make_golden.py [circle40 torus400 gauss8_120 batch512 diff256]

Takes minutes (torus400 alone: about 3 minutes on one core).
"""
from __future__ import annotations

import hashlib
import json
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
import pointclouds as pc  # noqa: E402

OUT = Path(__file__).resolve().parent


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def canonical(low, dims):
    pairs, ess = oracle.pairs_and_essential(low, dims)
    order = np.lexsort((pairs[:, 0], pairs[:, 1])) if len(pairs) else np.zeros(0, int)
    return pairs[order].astype(np.int64), np.sort(ess).astype(np.int64)


def one_cloud(coords, max_dim, max_diam2=-1):
    K = oracle.vr_build(coords, max_dim, max_diam2)
    r = oracle.reduce_pms(K)
    assert r.converged
    low_t, _ = oracle.reduce_twist(K)
    assert np.array_equal(low_t, r.low), "Algorithm 2 and Algorithm 3 disagree"
    pairs, ess = canonical(r.low, K["dim"])
    maxd = max_dim
    return dict(
        m=int(K.m),
        per_dim=np.bincount(K["dim"], minlength=maxd + 1).tolist(),
        n_pairs=int(len(pairs)),
        pairs_per_dim=np.bincount(K["dim"][pairs[:, 0]], minlength=maxd + 1).tolist()
        if len(pairs) else [0] * (maxd + 1),
        ess_per_dim=np.bincount(K["dim"][ess], minlength=maxd + 1).tolist(),
        pairs_sha=sha(pairs), ess_sha=sha(ess),
        passes=int(r.passes), pass_stats=r.stats[:, :8].tolist(),
    ), pairs, ess


def main(names):
    for name in names:
        t0 = time.time()
        if name == "circle40":
            x = pc.circle40()
            g, _, _ = one_cloud(x, 2)
        elif name == "torus400":
            x = pc.torus400()
            g, _, _ = one_cloud(x, 2)
        elif name == "gauss8_120":
            x = pc.gauss8_120()
            g, _, _ = one_cloud(x, 3, pc.GAUSS8_MAX_DIAM2)
            g["max_diam2"] = pc.GAUSS8_MAX_DIAM2
        elif name == "batch512":
            x, off = pc.batch512()
            clouds = []
            agg = None
            h = hashlib.sha256()
            for c in range(len(off) - 1):
                gc, pairs, ess = one_cloud(x[off[c]:off[c + 1]], 2)
                h.update(pairs.tobytes())
                h.update(ess.tobytes())
                st = np.array(gc.pop("pass_stats"), np.int64)
                agg = st if agg is None else (np.pad(agg, ((0, max(0, len(st) - len(agg))), (0, 0)))
                                              + np.pad(st, ((0, max(0, len(agg) - len(st))), (0, 0))))
                clouds.append(dict(m=gc["m"], n_pairs=gc["n_pairs"], passes=gc["passes"],
                                   pairs_sha=gc["pairs_sha"], ess_sha=gc["ess_sha"]))
            g = dict(m=int(sum(c["m"] for c in clouds)), n_clouds=len(clouds),
                     all_sha=h.hexdigest(), passes=int(max(c["passes"] for c in clouds)),
                     pass_stats=agg.tolist(), clouds=clouds)
            g["offsets_sha"] = sha(off)
        elif name == "diff256":
            # the differentiable form: fp32 clouds, pairing from the grid copy, loss over the
            # H1 pairs with fp64 Euclidean lengths of the realising edges
            x, off = pc.diff256()
            clouds = []
            for c in range(len(off) - 1):
                x64 = x[off[c]:off[c + 1]].astype(np.float64)
                K = oracle.vr_build(pc.to_grid(x64), 2)
                low, _ = oracle.reduce_twist(K)
                pairs, ess = canonical(low, K["dim"])
                edges = oracle.diagram_edges(K, low, 1)
                loss, grad = oracle.diagram_loss_grad(x64, edges)
                clouds.append(dict(m=int(K.m), n_pairs=int(len(pairs)), n_h1=int(len(edges)),
                                   pairs_sha=sha(pairs), ess_sha=sha(ess), loss=float(loss),
                                   grad_maxabs=float(np.abs(grad).max()),
                                   grad_l1=float(np.abs(grad).sum())))
            g = dict(m=int(sum(c["m"] for c in clouds)), n_clouds=len(clouds), dim=1,
                     loss_total=float(sum(c["loss"] for c in clouds)), clouds=clouds,
                     offsets_sha=sha(off))
        else:
            raise SystemExit(f"unknown workload {name}")
        g["coords_sha"] = sha(x)
        g["seconds_oracle"] = round(time.time() - t0, 1)
        g["generated_by"] = "tests/golden/make_golden.py (oracle only)"
        (OUT / f"{name}.json").write_text(json.dumps(g, indent=1) + "\n")
        print(name, g["m"], g.get("passes"), g["seconds_oracle"], "s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["circle40", "torus400", "gauss8_120", "batch512", "diff256"])
