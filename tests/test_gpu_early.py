"""Early-stopping quality curves (Sec. 4.2-4.4) from the device against the oracle's pass loop.

`early.profile` reruns the reduction with max_passes = l for every l; each state must equal the
oracle's state after the same passes, so the curves agree exactly. They also obey the
invariants the paper relies on: low never increases and stays >= lowstar (Thm 5), so the l1
error and the unreduced share only fall; E^l only shrinks and contains Ess (Lemma 11), so
its precision only rises; at convergence all three are exact.
"""
import numpy as np
import pytest

import pointclouds as pc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_04710_gb300 import build

    build.build()
    import oracle
    import paper_1708_04710_gb300 as ph

    oracle.build_lib()
    return torch, ph, oracle


@pytest.mark.parametrize("name,strict", [("gaussian15", False), ("trefoil15", True),
                                         ("sphere_product15", False)])
def test_profile_matches_oracle(env, name, strict):
    torch, ph, orc = env
    from paper_1708_04710_gb300 import early

    x = pc.ensemble15(name)
    ctx = ph.Context(collect_stats=True, strict_phase2=strict)
    ctx.build_filtration(torch.from_numpy(x).cuda(), None, 5)
    prof = early.profile(ctx)
    K = orc.vr_build(x, 5)
    assert prof["m"] == K.m == 9948  # complete 5-skeleton on 15 points
    full = orc.reduce_pms(K, strict=strict)
    assert prof["passes"] == full.passes
    for l in range(full.passes + 1):
        r = orc.reduce_pms(K, max_passes=l, strict=strict)
        assert prof["l1_error"][l] == early.relative_l1_error(r.low, full.low)
        assert prof["unreduced"][l] == early.unreduced_fraction(r.low, full.low)
        assert prof["precision"][l] == early.essential_precision(r.ess_est, full.ess_est)
        assert prof["adds"][l] == int(full.stats[:l, 6].sum())
        assert prof["xors"][l] == int(full.stats[:l, 7].sum())
    l1, un, pr = (np.array(prof[k]) for k in ("l1_error", "unreduced", "precision"))
    assert np.all(np.diff(l1) <= 0) and np.all(np.diff(un) <= 0) and np.all(np.diff(pr) >= 0)
    assert l1[-1] == 0 and un[-1] == 0 and pr[-1] == 1
    assert early.iterations_to(list(pr), [1.0], below=False)[1.0] <= full.passes
