"""Early stopping with Algorithm 2: how good the state is after a few iterations (Sec. 4).

The paper measures four things per iteration l of its outer loop:
- the relative l1 error of low^l against lowstar (Eq. rel_error);
- the proportion of columns not yet reduced, i.e. low^l(j) != lowstar(j);
- the precision |Ess| / |E^l| of the essential estimate (Eq. essential_iteration, Lemma 11);
- the cumulative column additions and XORs (Sec. 4.1).

`profile` reads each iteration's state from the device. Every pass is deterministic, so
rerunning the reduction from the unreduced matrix with max_passes = l gives exactly the state
after l iterations. That state is l passes with additions, followed by the marks and clearing
of pass l + 1, which the capped pass applies without additions. The functions here only do
arithmetic on the small host arrays read back; all reduction work runs in the library's
kernels.
"""
from __future__ import annotations

import numpy as np


def relative_l1_error(low: np.ndarray, lowstar: np.ndarray) -> float:
    """||low - lowstar||_1 / ||lowstar||_1 in the paper's 1-based indices (0 = no low)."""
    a = np.asarray(low, np.int64) + 1
    b = np.asarray(lowstar, np.int64) + 1
    den = np.abs(b).sum()
    return float(np.abs(a - b).sum() / den) if den else 0.0


def unreduced_fraction(low: np.ndarray, lowstar: np.ndarray) -> float:
    """Share of columns whose low is not yet lowstar."""
    low, lowstar = np.asarray(low), np.asarray(lowstar)
    return float(np.count_nonzero(low != lowstar) / max(len(low), 1))


def essential_precision(in_e: np.ndarray, ess: np.ndarray) -> float:
    """TP / (TP + FP) = |Ess| / |E^l|, using Ess subset of E^l (Lemma 11)."""
    n_e = int(np.count_nonzero(in_e))
    return float(np.count_nonzero(ess) / n_e) if n_e else 1.0


def profile(ctx, max_iterations: int | None = None) -> dict:
    """Per-iteration early-stopping quality of the filtration held by `ctx` (cloud 0).

    `ctx` is a library Context with a built filtration and collect_stats on. The result has one
    entry per iteration l = 0..L (L = passes of the full reduction, or max_iterations), each
    a list: l1_error, unreduced, precision (of E^l), and cumulative adds and xors up to l.
    """
    ctx.reset_reduction()
    full = ctx.reduce()
    if not full["converged"]:
        raise RuntimeError("the full reduction did not converge")
    lowstar = ctx.filtration(0)["low"]
    ess = ctx.essential_estimate(0)  # exact once converged: E = Ess
    stats = ctx.pass_stats()
    passes = full["passes"]
    last = passes if max_iterations is None else min(passes, max_iterations)
    adds = np.cumsum(stats[:, 6])
    xors = np.cumsum(stats[:, 7])
    out = {"passes": passes, "m": int(len(lowstar)), "ess": int(np.count_nonzero(ess)),
           "l1_error": [], "unreduced": [], "precision": [], "adds": [], "xors": []}
    for l in range(last + 1):
        ctx.reset_reduction()
        ctx.reduce(max_passes=l)
        low = ctx.filtration(0)["low"]
        out["l1_error"].append(relative_l1_error(low, lowstar))
        out["unreduced"].append(unreduced_fraction(low, lowstar))
        out["precision"].append(essential_precision(ctx.essential_estimate(0), ess))
        out["adds"].append(int(adds[l - 1]) if l > 0 else 0)
        out["xors"].append(int(xors[l - 1]) if l > 0 else 0)
    ctx.reset_reduction()
    ctx.reduce()
    return out


def iterations_to(values, levels, below: bool = True) -> dict:
    """First iteration at which a per-iteration curve reaches each level: the value is at or
    below the level (errors, unreduced share), or at or above it (precision)."""
    res = {}
    for lv in levels:
        hit = [i for i, v in enumerate(values) if (v <= lv if below else v >= lv)]
        res[lv] = hit[0] if hit else None
    return res
