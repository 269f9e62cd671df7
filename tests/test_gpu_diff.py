"""Differentiable diagrams on the GPU against the FP64 oracle, through the C ABI.

The pairing is integer work and must match exactly (same pairs, hence the same realising
edges); losses and gradients are FP32 on the GPU and FP64 in the oracle, compared normwise at
relative tolerance 1e-4: max |g_gpu - g_ref| <= 1e-4 * max |g_ref|. The oracle's gradient is
itself pinned by FP64 central differences in test_oracle_pins.py.
"""
import math

import numpy as np
import pytest

import pointclouds as pc

pytestmark = pytest.mark.gpu
RTOL = 1e-4


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


def _oracle(orc, x32, dim):
    x64 = x32.astype(np.float64)
    K = orc.vr_build(pc.to_grid(x64), dim + 1)
    low = orc.reduce_twist(K)[0]
    edges = orc.diagram_edges(K, low, dim)
    loss, grad = orc.diagram_loss_grad(x64, edges)
    return loss, grad, len(edges)


@pytest.mark.parametrize("dim", [0, 1])
def test_single_cloud_loss_and_gradient(env, dim):
    torch, ph, orc = env
    rng = np.random.Generator(np.random.PCG64(5))
    x = pc.sphere(40, rng, noise=0.02).astype(np.float32)
    ctx = ph.Context()
    xt = torch.from_numpy(x).cuda()
    ctx.build_filtration_f32(xt, None, dim + 1)
    assert ctx.reduce()["converged"]
    loss = ctx.diagram_loss(xt, dim).cpu().numpy()
    grad = ctx.diagram_backward(xt, torch.ones(1, device="cuda"), dim).cpu().numpy()
    ref_loss, ref_grad, npairs = _oracle(orc, x, dim)
    assert ctx.last_pairs == npairs
    assert abs(loss[0] - ref_loss) <= RTOL * abs(ref_loss)
    assert loss[1] == loss[0]
    assert np.abs(grad - ref_grad).max() <= RTOL * np.abs(ref_grad).max()


def test_batched_autograd_matches_oracle(env):
    torch, ph, orc = env
    from paper_1708_04710_gb300.diff import diagram_loss

    x, off = pc.diff256(n_clouds=12)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    w = torch.linspace(0.5, 1.5, 12, device="cuda")
    per_cloud = diagram_loss(xt, off, dim=1)
    (per_cloud * w).sum().backward()
    got_loss = per_cloud.detach().cpu().numpy()
    got_grad = xt.grad.cpu().numpy()
    ref_grad = np.zeros_like(got_grad, dtype=np.float64)
    for c in range(12):
        a, b = off[c], off[c + 1]
        loss, g, npairs = _oracle(orc, x[a:b], 1)
        assert npairs == math.comb(64, 2) - 63  # complete 2-skeleton: every cycle dies
        assert abs(got_loss[c] - loss) <= RTOL * loss
        ref_grad[a:b] = w[c].item() * g
    assert np.abs(got_grad - ref_grad).max() <= RTOL * np.abs(ref_grad).max()


def test_full_diff256_properties_and_samples(env):
    torch, ph, orc = env
    x, off = pc.diff256()
    xt = torch.from_numpy(x).cuda()
    ctx = ph.Context()
    ctx.build_filtration_f32(xt, off, 2)
    assert ctx.m == 256 * (64 + math.comb(64, 2) + math.comb(64, 3))
    assert ctx.reduce()["converged"]
    loss = ctx.diagram_loss(xt, 1)
    assert ctx.last_pairs == 256 * (math.comb(64, 2) - 63)
    grad = ctx.diagram_backward(xt, torch.ones(256, device="cuda"), 1).cpu().numpy()
    lc = loss.cpu().numpy()
    assert abs(lc[-1] - lc[:-1].astype(np.float64).sum()) <= 1e-5 * lc[-1]
    # translation invariance: every cloud's gradient sums to zero
    for c in range(256):
        gsum = grad[off[c]:off[c + 1]].sum(0)
        assert np.abs(gsum).max() <= 1e-4 * np.abs(grad[off[c]:off[c + 1]]).max()
    # sampled clouds against the oracle
    for c in (0, 77, 255):
        a, b = off[c], off[c + 1]
        ref_loss, ref_grad, _ = _oracle(orc, x[a:b], 1)
        assert abs(lc[c] - ref_loss) <= RTOL * ref_loss
        assert np.abs(grad[a:b] - ref_grad).max() <= RTOL * np.abs(ref_grad).max()


def test_rejects_bad_input(env):
    torch, ph, _ = env
    ctx = ph.Context()
    bad = torch.tensor([[0.0, 1.0], [float("nan"), 0.0]], device="cuda")
    with pytest.raises(ph.PHError):
        ctx.build_filtration_f32(bad, None, 2)
    ctx.load_boundary(np.array([0, 0, 1], np.int32), np.array([0, 0, 0, 2], np.int64),
                      np.array([0, 1], np.int32))
    ctx.reduce()
    with pytest.raises(ph.PHError):  # a loaded complex has no coordinates
        ctx.diagram_loss(torch.zeros((2, 2), device="cuda"), 0)
