"""Bytes moved between ranks by the single-filtration exchange, measured on CPU gloo ranks.

    python tests/exchange_volume.py 60 2      # first 60 torus points, 2 ranks

Builds the complete Vietoris-Rips complex up to triangles of the first n torus points with the
oracle, reduces it over k gloo ranks with the numpy shard of ``shard_cpu.py`` and prints one
JSON line: tables sent in a pass (all ranks, the median over the passes), source-column bytes
over the reduction and in its largest pass, and the method's addition bytes (8 B per
nontrivial XOR) for comparison.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path[:0] = [os.path.dirname(HERE), HERE]


def main():
    import oracle
    import pointclouds as pc
    from test_sharded_exchange import _run_ranks

    n, world = int(sys.argv[1]), int(sys.argv[2])
    oracle.build_lib()
    K = oracle.vr_build(pc.torus400(n), 2)
    (_, res, _, _), = _run_ranks(world, [(f"torus{n}", K, oracle.beta(K), {})])[0]
    st, moved = res["stats"], res["exchange"]
    print(json.dumps({
        "points": n, "ranks": world, "m": K.m, "table_rows": int((K["dim"] < 2).sum()),
        "passes": int(res["passes"]), "table_bytes_per_pass": float(np.median(moved[:, 0])),
        "column_bytes": int(moved[:, 1].sum()), "column_bytes_largest_pass": int(moved[:, 1].max()),
        "addition_bytes": 8 * int(st[:, 7].sum())}))


if __name__ == "__main__":
    main()
