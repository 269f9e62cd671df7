"""Differentiable diagrams on the GPU against the FP64 oracle, through the C ABI.

The pairing is integer work and must match exactly (same pairs, hence the same realising
edges); losses and gradients are FP32 on the GPU and FP64 in the oracle, compared at relative
tolerance 1e-4, normwise (max |g_gpu - g_ref| <= 1e-4 * max |g_ref|) and element by element:

    |g_gpu - g_ref| <= 1e-4 * |g_ref| + 16 u * max |g_ref|   (per cloud, u = 2^-24).

The second term is for components near zero, where a relative bound means nothing: each
gradient component is an FP32 sum, in atomic (arbitrary) order, of about 125 pair terms whose
magnitudes exceed the result, so its rounding error is a few units in the last place of the
cloud's largest component (an FP32 emulation of the kernel's arithmetic, in random order,
stays below 4.4 u * max |g_ref| on diff256), not a fraction of the component itself. The
oracle's gradient is itself pinned by FP64 central differences in test_oracle_pins.py.
"""
import hashlib
import json
import math
from pathlib import Path

import numpy as np
import pytest

import pointclouds as pc

pytestmark = pytest.mark.gpu
RTOL = 1e-4
ULP_FLOOR = 16 * 2.0 ** -24  # times the cloud's largest gradient component
GOLDEN = Path(__file__).resolve().parent / "golden" / "diff256.json"


def _elementwise_ok(got, ref):
    """The element-wise rule of the module docstring; returns (ok, worst ratio to the bound)."""
    bound = RTOL * np.abs(ref) + ULP_FLOOR * np.abs(ref).max()
    ratio = float((np.abs(got - ref) / bound).max()) if ref.size else 0.0
    return ratio <= 1.0, ratio


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
    assert _elementwise_ok(grad, ref_grad)[0]


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
        assert _elementwise_ok(got_grad[a:b], ref_grad[a:b])[0], c
    assert np.abs(got_grad - ref_grad).max() <= RTOL * np.abs(ref_grad).max()


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def test_full_diff256_every_cloud(env):
    """The full differentiable workload (256 clouds x 64 points, 11.2M simplices): every
    cloud's pairs and essentials bit-exact against the oracle's stored SHA-256, every cloud's
    loss against the stored FP64 loss, and every gradient component against the oracle's FP64
    gradient (element-wise rule above), the oracle run live on all 256 clouds."""
    torch, ph, orc = env
    g = json.loads(GOLDEN.read_text())
    x, off = pc.diff256()
    assert _sha(off) == g["offsets_sha"] and _sha(x) == g["coords_sha"], "generator drift"
    xt = torch.from_numpy(x).cuda()
    ctx = ph.Context()
    ctx.build_filtration_f32(xt, off, 2)
    assert ctx.m == 256 * (64 + math.comb(64, 2) + math.comb(64, 3)) == g["m"]
    assert ctx.reduce()["converged"]
    loss = ctx.diagram_loss(xt, 1)
    assert ctx.last_pairs == 256 * (math.comb(64, 2) - 63)
    grad = ctx.diagram_backward(xt, torch.ones(256, device="cuda"), 1).cpu().numpy()
    lc = loss.cpu().numpy()
    assert abs(lc[-1] - g["loss_total"]) <= RTOL * g["loss_total"]
    worst = 0.0
    for c in range(256):
        gc = g["clouds"][c]
        pr = ctx.pairs(c, on_device=False)
        es = ctx.essential(c, on_device=False)
        b, d = pr["birth"].numpy(), pr["death"].numpy()
        o = np.lexsort((b, d))
        pairs = np.stack([b[o], d[o]], 1).astype(np.int64)
        assert _sha(pairs) == gc["pairs_sha"], f"cloud {c}: pairs differ from the oracle"
        assert _sha(np.sort(es["idx"].numpy()).astype(np.int64)) == gc["ess_sha"], c
        assert abs(lc[c] - gc["loss"]) <= RTOL * gc["loss"], c
        a, e = off[c], off[c + 1]
        ref_loss, ref_grad, n_h1 = _oracle(orc, x[a:e], 1)
        # the live oracle is the one that wrote the golden values
        assert n_h1 == gc["n_h1"] and abs(ref_loss - gc["loss"]) <= 1e-9 * gc["loss"], c
        assert abs(np.abs(ref_grad).max() - gc["grad_maxabs"]) <= 1e-9 * gc["grad_maxabs"], c
        ok, ratio = _elementwise_ok(grad[a:e], ref_grad)
        worst = max(worst, ratio)
        assert ok, f"cloud {c}: gradient off by {ratio:.2f} of the element-wise bound"
        assert np.abs(grad[a:e] - ref_grad).max() <= RTOL * np.abs(ref_grad).max(), c
        # translation invariance: each cloud's gradient sums to zero
        assert np.abs(grad[a:e].sum(0)).max() <= 1e-4 * np.abs(grad[a:e]).max(), c
    print(f"diff256: worst gradient error {worst:.3f} of the element-wise bound")


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


def test_diagram_calls_reject_wrong_shapes_before_any_launch(env):
    """The diagram kernels index the coordinates by the build's point rows, so a wrong D or a
    coordinate array of another shape must be refused before anything is launched."""
    import ctypes

    torch, ph, _ = env
    x, off = pc.diff256(n_clouds=2)
    xt = torch.from_numpy(x).cuda()
    ctx = ph.Context()
    ctx.build_filtration_f32(xt, off, 2)
    assert ctx.reduce()["converged"]
    lib = ph.load_library()
    loss = torch.zeros(3, device="cuda")
    grad = torch.zeros_like(xt)
    gl = torch.ones(2, device="cuda")
    n = ctypes.c_int64(0)
    before = ctx.kernel_launches()
    rc = lib.ph_diagram_loss(ctx._h, ctypes.c_void_p(xt.data_ptr()), 2, 1,
                             ctypes.c_void_p(loss.data_ptr()), ctypes.byref(n))
    assert rc == -1 and b"D must equal" in lib.ph_last_error(ctx._h)  # PH_ERR_INVALID
    rc = lib.ph_diagram_backward(ctx._h, ctypes.c_void_p(xt.data_ptr()), 4, 1,
                                 ctypes.c_void_p(gl.data_ptr()), ctypes.c_void_p(grad.data_ptr()))
    assert rc == -1
    assert ctx.kernel_launches() == before
    # the binding checks the whole shape (it knows N): fewer points, or another D
    for bad in (xt[:-1], xt[:, :2], xt.double()):
        with pytest.raises(ph.PHError):
            ctx.diagram_loss(bad, 1)
        with pytest.raises(ph.PHError):
            ctx.diagram_backward(bad, gl, 1)
    with pytest.raises(ph.PHError):  # one upstream value per cloud
        ctx.diagram_backward(xt, torch.ones(3, device="cuda"), 1)
    assert ctx.kernel_launches() == before
    assert torch.isfinite(ctx.diagram_loss(xt, 1)).all()


def test_autograd_refuses_a_rebuilt_context(env):
    """Two losses on one context: the first loss's backward would scatter through the second
    filtration's pairing, so it raises instead."""
    torch, ph, _ = env
    from paper_1708_04710_gb300.diff import diagram_loss

    x, off = pc.diff256(n_clouds=2)
    shared = ph.Context()
    xa = torch.from_numpy(x).cuda().requires_grad_(True)
    xb = (torch.from_numpy(x).cuda() * 1.01).requires_grad_(True)
    la = diagram_loss(xa, off, 1, shared).sum()
    lb = diagram_loss(xb, off, 1, shared).sum()
    lb.backward()  # the context's current filtration: fine
    with pytest.raises(RuntimeError, match="rebuilt"):
        la.backward()
