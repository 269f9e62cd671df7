"""The allocation-free beta entry point agrees with the allocating path, through the C ABI.

ph_beta_static serves callers that cannot allocate device memory -- code living inside another
framework's memory pool, programs that forbid allocation after start-up, callers without a
library context. Its scratch is a fixed device array shared by every call, so this test makes
several calls in a row, each with a different size, and checks each result against beta read
back from a context built by ph_build_filtration (which allocates its own scratch), and against
the oracle.
"""
import ctypes

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


def _local_rows(K, d):
    """Boundary rows of the dimension-d columns as positions inside dimension d-1."""
    dims = K["dim"]
    pos = np.full(K.m, -1, np.int64)
    for e in range(dims.max() + 1):
        idx = np.nonzero(dims == e)[0]
        pos[idx] = np.arange(len(idx))
    cols = np.nonzero(dims == d)[0]
    rows = np.stack([K["rows"][K["colptr"][j]:K["colptr"][j + 1]] for j in cols])
    return pos[rows].astype(np.int32), cols, pos


def _pool_used(torch):
    """Bytes in use in the device's default memory pool (what cudaMallocAsync draws from), or
    None where the CUDA runtime library cannot be opened from Python."""
    import ctypes.util

    for name in ("libcudart.so", "libcudart.so.13", ctypes.util.find_library("cudart")):
        try:
            rt = ctypes.CDLL(name or "libcudart.so")
            break
        except OSError:
            rt = None
    if rt is None:
        return None
    pool = ctypes.c_void_p()
    if rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) != 0:
        return None
    used = ctypes.c_uint64()
    attr_used_mem_current = 7  # cudaMemPoolAttrUsedMemCurrent
    if rt.cudaMemPoolGetAttribute(pool, attr_used_mem_current, ctypes.byref(used)) != 0:
        return None
    return used.value


def test_beta_static_matches_allocating_path(env):
    torch, ph, oracle = env
    lib = ph.load_library()
    x = pc.gauss8_120()[:70]
    cut = pc.GAUSS8_MAX_DIAM2
    K = oracle.vr_build(x, 3, cut)
    ctx = ph.Context()
    ctx.build_filtration(torch.from_numpy(x).cuda(), None, 3, cut)
    beta_ctx = ctx.filtration(0)["beta"]  # filtration indices, from the allocating path
    beta_orc = oracle.beta(K)
    assert np.array_equal(beta_ctx, beta_orc)
    stream = torch.cuda.current_stream()
    inputs = {}
    for d in (1, 2, 3):  # every buffer the calls use exists before the first call
        rows, cols, pos = _local_rows(K, d)
        inputs[d] = (rows, cols, pos, torch.from_numpy(rows).cuda(),
                     torch.full((len(cols),), -7, dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    torch_allocs = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    pool0 = _pool_used(torch)
    # several calls in a row, large then small then large again: leftovers must not leak
    for d in (3, 1, 2, 3, 1):
        rows, cols, pos, r_dev, out = inputs[d]
        n_rows = int((K["dim"] == d - 1).sum())
        out.fill_(-7)
        rc = lib.ph_beta_static(ctypes.c_void_p(r_dev.data_ptr()), len(cols), d + 1, n_rows,
                                ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        got = out.cpu().numpy()
        expect = np.where(beta_ctx[cols] >= 0, pos[np.maximum(beta_ctx[cols], 0)], -1)
        assert np.array_equal(got, expect), d
    # nothing was allocated on the device meanwhile: not through torch's allocator, and not
    # from the default memory pool (the GPU is shared, so device-wide free memory says nothing)
    torch.cuda.synchronize()
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == torch_allocs
    if pool0 is not None:
        assert _pool_used(torch) == pool0


def test_beta_static_rejects_oversize_and_bad_rows(env):
    torch, ph, _ = env
    lib = ph.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rows = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    out = torch.empty(4, dtype=torch.int32, device="cuda")
    assert lib.ph_beta_static(ctypes.c_void_p(rows.data_ptr()), 4, 2, (1 << 22) + 1,
                              ctypes.c_void_p(out.data_ptr()), stream) == -4  # PH_ERR_CAPACITY
    rows[1, 1] = 9  # outside [0, n_rows)
    assert lib.ph_beta_static(ctypes.c_void_p(rows.data_ptr()), 4, 2, 5,
                              ctypes.c_void_p(out.data_ptr()), stream) == -1  # PH_ERR_INVALID
    rows[1, 1] = 3
    assert lib.ph_beta_static(ctypes.c_void_p(rows.data_ptr()), 4, 2, 5,
                              ctypes.c_void_p(out.data_ptr()), stream) == 0
    # rows 0 and 3 first appear in column 0 and column 1 respectively
    assert out.cpu().tolist() == [0, 3, -1, -1]
