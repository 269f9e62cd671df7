"""ctypes binding of the C ABI in ``include/ph_gb300.h``: argument marshalling only.

Every computation runs in the CUDA library ``libph_gb300.so``. PyTorch supplies device memory
(through its caching allocator, handed to the library as a ``ph_allocator``) and the stream.
There is no fallback: if the library is missing or no GPU is present, loading fails loudly.
"""
from __future__ import annotations

import os

import ctypes
from ctypes import (CFUNCTYPE, POINTER, Structure, byref, c_char_p, c_double, c_int, c_int32,
                    c_int64, c_size_t, c_void_p)
from pathlib import Path

import numpy as np

# PH_GB300_DEBUG=1: the build with device-side bounds checks (build.build(debug=True))
LIB_PATH = Path(__file__).resolve().parent / (
    "libph_gb300_debug.so" if os.environ.get("PH_GB300_DEBUG") == "1" else "libph_gb300.so")

PH_OK, PH_NOT_CONVERGED = 0, 1
PS_FIELDS = ("active", "new_pivots", "zero_final", "cor10", "cleared", "targets", "adds",
             "xors", "copied", "ess_est", "predicted", "empty_l", "packed")


class PHError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ph error {code}: {msg}")
        self.code = code


class PhOpts(Structure):
    _fields_ = [("strict_phase2", c_int32), ("use_cor10", c_int32), ("lane_merge_words", c_int32),
                ("staged_merge_max", c_int32), ("merge_items", c_int32),
                ("collect_stats", c_int32), ("use_graph", c_int32), ("time_kernels", c_int32),
                ("add_blocks_per_sm", c_int32), ("timeout_ms", c_int32),
                ("predict_pairs", c_int32), ("dense_threshold", c_int32),
                ("warp_chunks_below", c_int32), ("warp_chunk_words", c_int32),
                ("narrow_chunks_below", c_int32), ("phase2_sets", c_int32),
                ("phase2_priority", c_int32), ("arena_words", c_int64)]


class PhStats(Structure):
    _fields_ = [("passes", c_int32), ("status", c_int32), ("m", c_int64), ("col_adds", c_int64),
                ("xors", c_int64), ("alg_bytes", c_int64), ("add_bytes", c_int64),
                ("add_launches", c_int64), ("ms_add", c_double)]


ALLOC_FN = CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)


class PhAllocator(Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", c_void_p)]


# exported symbols and their signatures: the ABI the tests check against include/ph_gb300.h
SIGNATURES = {
    "ph_default_opts": (None, [POINTER(PhOpts)]),
    "ph_create": (c_int, [POINTER(c_void_p), POINTER(PhOpts), POINTER(PhAllocator), c_void_p]),
    "ph_destroy": (None, [c_void_p]),
    "ph_build_filtration": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_int32,
                                    c_int32, c_int64, POINTER(c_int64)]),
    "ph_build_filtration_f32": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int64,
                                        c_int32, c_int32, c_int64, POINTER(c_int64)]),
    "ph_build_filtration_scales": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int64,
                                           c_int32, c_int32, c_int64, c_int32,
                                           POINTER(c_int64)]),
    "ph_load_boundary": (c_int, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "ph_diagram_loss": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_void_p,
                                POINTER(c_int64)]),
    "ph_diagram_backward": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p]),
    "ph_reduce": (c_int, [c_void_p, c_int32, POINTER(PhStats)]),
    "ph_reset_reduction": (c_int, [c_void_p]),
    "ph_get_pass_stats": (c_int, [c_void_p, c_void_p, c_int32, POINTER(c_int32)]),
    "ph_get_pairs": (c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                             c_int64, POINTER(c_int64), c_int32]),
    "ph_get_essential": (c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_int64,
                                 POINTER(c_int64), c_int32]),
    "ph_get_filtration": (c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p, POINTER(c_int64)]),
    "ph_beta_static": (c_int, [c_void_p, c_int64, c_int32, c_int64, c_void_p, c_void_p]),
    "ph_get_add_times": (c_int, [c_void_p, c_void_p, c_int32, POINTER(c_int32)]),
    "ph_get_essential_estimate": (c_int, [c_void_p, c_int32, c_void_p, POINTER(c_int64)]),
    "ph_get_predicted_lows": (c_int, [c_void_p, c_int32, c_void_p, POINTER(c_int64)]),
    "ph_get_columns": (c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_int64,
                               POINTER(c_int64)]),
    "ph_kernel_launches": (c_int64, [c_void_p]),
    "ph_last_error": (c_char_p, [c_void_p]),
}

_lib = None


def load_library(path: Path | str = LIB_PATH):
    """Loads the CUDA library; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = Path(path)
    if not path.exists():
        raise ImportError(f"{path} is missing: run __graft_entry__.build() (or "
                          "python paper_1708_04710_gb300/build.py) first")
    lib = ctypes.CDLL(str(path))
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("the persistent-homology library needs a CUDA GPU")
    return torch


def _ptr(t) -> c_void_p:
    if t is None:
        return c_void_p(None)
    if isinstance(t, np.ndarray):
        return c_void_p(t.ctypes.data)
    return c_void_p(t.data_ptr())


class Context:
    """One library context: a filtration (of one or many clouds) and its reduction."""

    def __init__(self, *, strict_phase2: bool = False, use_cor10: bool = True,
                 collect_stats: bool = False, staged_merge_max: int = 0, merge_items: int = 0,
                 use_graph: bool = True, time_kernels: bool = False, add_blocks_per_sm: int = 0,
                 timeout_ms: int = 0, predict_pairs: bool = False, dense_threshold: int = 0,
                 warp_chunks_below: int = 0, warp_chunk_words: int = 0, lane_merge_words: int = 0,
                 narrow_chunks_below: int = 0, phase2_sets: int = 0,
                 phase2_priority: int = 0,
                 arena_words: int = 0,
                 stream=None, device_alloc=None, device_free=None):
        torch = _torch()
        self._torch = torch
        self.lib = load_library()
        opts = PhOpts()
        self.lib.ph_default_opts(byref(opts))
        opts.strict_phase2 = int(strict_phase2)
        opts.use_cor10 = int(use_cor10)
        opts.collect_stats = int(collect_stats)
        if staged_merge_max:
            opts.staged_merge_max = int(staged_merge_max)
        opts.merge_items = int(merge_items)
        opts.use_graph = int(use_graph)
        opts.time_kernels = int(time_kernels)
        opts.add_blocks_per_sm = int(add_blocks_per_sm)
        opts.timeout_ms = int(timeout_ms)
        opts.predict_pairs = int(predict_pairs)
        opts.dense_threshold = int(dense_threshold)
        opts.warp_chunks_below = int(warp_chunks_below)
        opts.warp_chunk_words = int(warp_chunk_words)
        opts.lane_merge_words = int(lane_merge_words)
        opts.narrow_chunks_below = int(narrow_chunks_below)
        opts.phase2_sets = int(phase2_sets)
        opts.phase2_priority = int(phase2_priority)
        opts.arena_words = int(arena_words)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self.stream.device
        dev_index = self.device.index if self.device.index is not None else 0

        # device memory: torch's caching allocator, or the caller's device_alloc(nbytes, stream)
        # -> pointer (0 / None: out of memory) and device_free(pointer)
        def _alloc(nbytes, user, stream):
            try:
                if device_alloc is not None:
                    return device_alloc(int(nbytes), stream or 0) or None
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev_index, stream or 0)
            except Exception:  # out of memory: the library reports PH_ERR_ALLOC
                return None

        def _free(ptr, nbytes, user, stream):
            if device_free is not None:
                device_free(ptr)
            else:
                torch.cuda.caching_allocator_delete(ptr)

        self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))  # keep the callbacks alive
        self._allocator = PhAllocator(self._cb[0], self._cb[1], None)
        self._h = c_void_p()
        with torch.cuda.device(self.device):
            self._check(self.lib.ph_create(byref(self._h), byref(opts), byref(self._allocator),
                                           c_void_p(self.stream.cuda_stream)))
        self.n_clouds = 0
        self.m = 0
        self.builds = 0        # filtrations built or loaded so far
        self._points = None    # (N, D) of the current VR build from float32 coordinates

    # -- helpers --------------------------------------------------------------------------
    def _check(self, rc: int) -> int:
        if rc < 0:
            msg = self.lib.ph_last_error(self._h).decode() if self._h else ""
            raise PHError(rc, msg)
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self.lib.ph_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- ABI ------------------------------------------------------------------------------
    def build_filtration(self, coords, cloud_offsets=None, max_dim: int = 2,
                         max_diam2: int = -1) -> int:
        """coords: int32 CUDA tensor (N, D) in grid units; cloud_offsets: int64 (n_clouds+1)."""
        torch = self._torch
        assert coords.is_cuda and coords.dtype == torch.int32 and coords.dim() == 2
        coords = coords.contiguous()
        self._coords = coords
        N, D = coords.shape
        if cloud_offsets is None:
            offs = None
            nc = 1
        else:
            offs = np.ascontiguousarray(np.asarray(cloud_offsets, dtype=np.int64))
            nc = len(offs) - 1
        m = c_int64(0)
        self._points = None
        self._check(self.lib.ph_build_filtration(self._h, _ptr(coords), _ptr(offs), nc, N, D,
                                                 max_dim, int(max_diam2), byref(m)))
        self.n_clouds = nc
        self.m = m.value
        self.builds += 1
        return self.m

    def build_filtration_scales(self, coords, cloud_offsets=None, max_dim: int = 2,
                                scale_step: int = 1, n_scales: int = 1) -> int:
        """Like build_filtration on a grid of scales r_i = i * scale_step (grid units),
        i = 0..n_scales: the filtration value of a simplex is its scale index."""
        torch = self._torch
        assert coords.is_cuda and coords.dtype == torch.int32 and coords.dim() == 2
        coords = coords.contiguous()
        self._coords = coords
        N, D = coords.shape
        offs = None if cloud_offsets is None else np.ascontiguousarray(
            np.asarray(cloud_offsets, dtype=np.int64))
        nc = 1 if offs is None else len(offs) - 1
        m = c_int64(0)
        self._points = None
        self._check(self.lib.ph_build_filtration_scales(self._h, _ptr(coords), _ptr(offs), nc, N,
                                                        D, max_dim, int(scale_step),
                                                        int(n_scales), byref(m)))
        self.n_clouds = nc
        self.m = m.value
        self.builds += 1
        return self.m

    def build_filtration_f32(self, coords, cloud_offsets=None, max_dim: int = 2,
                             max_diam2: int = -1) -> int:
        """coords: float32 CUDA tensor (N, D); rounded to the grid on the device."""
        torch = self._torch
        assert coords.is_cuda and coords.dtype == torch.float32 and coords.dim() == 2
        coords = coords.contiguous()
        N, D = coords.shape
        offs = None if cloud_offsets is None else np.ascontiguousarray(
            np.asarray(cloud_offsets, dtype=np.int64))
        nc = 1 if offs is None else len(offs) - 1
        m = c_int64(0)
        self._points = None
        self._check(self.lib.ph_build_filtration_f32(self._h, _ptr(coords), _ptr(offs), nc, N, D,
                                                     max_dim, int(max_diam2), byref(m)))
        self._points = (int(N), int(D))
        self.n_clouds = nc
        self.m = m.value
        self.builds += 1
        return self.m

    def _check_points(self, coords):
        """The diagram kernels index coords by the build's point rows: the tensor must be the
        float32 (N, D) CUDA array of the last build_filtration_f32."""
        if self._points is None:
            raise PHError(-1, "diagram losses need a filtration built by build_filtration_f32")
        if (not coords.is_cuda or coords.dtype != self._torch.float32
                or tuple(coords.shape) != self._points):
            raise PHError(-1, f"coords must be a float32 CUDA tensor of shape {self._points} "
                              f"(got {coords.dtype} {tuple(coords.shape)})")

    def diagram_loss(self, coords, dim: int = 1):
        """Per-cloud losses followed by their sum (float32 tensor, n_clouds + 1)."""
        torch = self._torch
        self._check_points(coords)
        coords = coords.contiguous()
        out = torch.empty(self.n_clouds + 1, dtype=torch.float32, device=coords.device)
        n = c_int64(0)
        self._check(self.lib.ph_diagram_loss(self._h, _ptr(coords), coords.shape[1], dim,
                                             _ptr(out), byref(n)))
        self.last_pairs = n.value
        return out

    def diagram_backward(self, coords, grad_loss, dim: int = 1, grad=None):
        torch = self._torch
        self._check_points(coords)
        coords = coords.contiguous()
        if grad is None:
            grad = torch.zeros_like(coords)
        elif (tuple(grad.shape) != tuple(coords.shape) or grad.dtype != torch.float32
              or not grad.is_contiguous() or grad.device != coords.device):
            raise PHError(-1, "grad must be a contiguous float32 tensor shaped like coords")
        g = grad_loss.contiguous().to(torch.float32)
        if g.numel() != self.n_clouds or not g.is_cuda:
            raise PHError(-1, f"grad_loss must hold one CUDA value per cloud ({self.n_clouds})")
        self._check(self.lib.ph_diagram_backward(self._h, _ptr(coords), coords.shape[1], dim,
                                                 _ptr(g), _ptr(grad)))
        return grad

    def load_boundary(self, dims, colptr, rows):
        dims = np.ascontiguousarray(dims, np.int32)
        colptr = np.ascontiguousarray(colptr, np.int64)
        rows = np.ascontiguousarray(rows, np.int32)
        self._points = None
        self._check(self.lib.ph_load_boundary(self._h, len(dims), _ptr(dims), _ptr(colptr),
                                              _ptr(rows)))
        self.n_clouds = 1
        self.m = len(dims)
        self.builds += 1

    def reduce(self, max_passes: int = -1) -> dict:
        st = PhStats()
        rc = self._check(self.lib.ph_reduce(self._h, max_passes, byref(st)))
        return dict(passes=st.passes, status=st.status, converged=(rc == PH_OK), m=st.m,
                    col_adds=st.col_adds, xors=st.xors, alg_bytes=st.alg_bytes,
                    add_bytes=st.add_bytes, add_launches=st.add_launches, ms_add=st.ms_add)

    def add_times(self) -> np.ndarray:
        n = c_int32(0)
        self._check(self.lib.ph_get_add_times(self._h, None, 0, byref(n)))
        out = np.zeros(n.value, np.float32)
        self._check(self.lib.ph_get_add_times(self._h, _ptr(out), n.value, byref(n)))
        return out

    def essential_estimate(self, cloud: int = 0) -> np.ndarray:
        """E^l after the passes run so far (Eq. essential_iteration), as a boolean mask over the
        cloud's simplices in filtration order; it contains every essential simplex."""
        n = c_int64(0)
        self._check(self.lib.ph_get_essential_estimate(self._h, int(cloud), None, byref(n)))
        out = np.zeros(n.value, np.uint8)
        self._check(self.lib.ph_get_essential_estimate(self._h, int(cloud), _ptr(out), byref(n)))
        return out.astype(bool)

    def predicted_lows(self, cloud: int = 0) -> np.ndarray:
        """lowstar predicted by Corollary 10 (non-zero case) per simplex of the cloud in
        filtration order (filtration index, -1 where none); needs predict_pairs."""
        n = c_int64(0)
        self._check(self.lib.ph_get_predicted_lows(self._h, int(cloud), None, byref(n)))
        out = np.zeros(n.value, np.int32)
        self._check(self.lib.ph_get_predicted_lows(self._h, int(cloud), _ptr(out), byref(n)))
        return out

    def columns(self, cloud: int = 0):
        """The reduced matrix R of the cloud as (colptr int64 [count + 1], rows int32), columns
        and rows as filtration indices: for a negative column j of a complete reduction, the
        rows of column j are a cycle representing the class born at low(j)."""
        n = c_int64(0)
        self._check(self.lib.ph_get_filtration(self._h, int(cloud), None, None, None, None,
                                               None, byref(n)))
        colptr = np.zeros(n.value + 1, np.int64)
        nnz = c_int64(0)
        self._check(self.lib.ph_get_columns(self._h, int(cloud), _ptr(colptr), None, 0,
                                            byref(nnz)))
        rows = np.zeros(max(nnz.value, 1), np.int32)
        self._check(self.lib.ph_get_columns(self._h, int(cloud), _ptr(colptr), _ptr(rows),
                                            nnz.value, byref(nnz)))
        return colptr, rows[:nnz.value]

    def kernel_launches(self) -> int:
        return int(self.lib.ph_kernel_launches(self._h))

    def reset_reduction(self):
        self._check(self.lib.ph_reset_reduction(self._h))

    def pass_stats(self) -> np.ndarray:
        rows = c_int32(0)
        self._check(self.lib.ph_get_pass_stats(self._h, None, 0, byref(rows)))
        out = np.zeros((rows.value, len(PS_FIELDS)), np.int64)
        self._check(self.lib.ph_get_pass_stats(self._h, _ptr(out), rows.value, byref(rows)))
        return out

    def pairs(self, cloud: int = 0, on_device: bool = True) -> dict:
        torch = self._torch
        n = c_int64(0)
        self._check(self.lib.ph_get_pairs(self._h, cloud, None, None, None, None, None, 0,
                                          byref(n), 0))
        k = n.value
        if on_device:
            mk = lambda dt: torch.empty(k, dtype=dt, device=self.device)  # noqa: E731
        else:  # page-locked, so the device-to-host copies run at full speed
            mk = lambda dt: torch.empty(k, dtype=dt, pin_memory=True)  # noqa: E731
        out = dict(birth=mk(torch.int64), death=mk(torch.int64), dim=mk(torch.int32),
                   birth_diam2=mk(torch.int64), death_diam2=mk(torch.int64))
        self._check(self.lib.ph_get_pairs(self._h, cloud, _ptr(out["birth"]), _ptr(out["death"]),
                                          _ptr(out["dim"]), _ptr(out["birth_diam2"]),
                                          _ptr(out["death_diam2"]), k, byref(n),
                                          int(on_device)))
        return out

    def essential(self, cloud: int = 0, on_device: bool = True) -> dict:
        torch = self._torch
        n = c_int64(0)
        self._check(self.lib.ph_get_essential(self._h, cloud, None, None, None, 0, byref(n), 0))
        k = n.value
        if on_device:
            mk = lambda dt: torch.empty(k, dtype=dt, device=self.device)  # noqa: E731
        else:  # page-locked, so the device-to-host copies run at full speed
            mk = lambda dt: torch.empty(k, dtype=dt, pin_memory=True)  # noqa: E731
        out = dict(idx=mk(torch.int64), dim=mk(torch.int32), diam2=mk(torch.int64))
        self._check(self.lib.ph_get_essential(self._h, cloud, _ptr(out["idx"]), _ptr(out["dim"]),
                                              _ptr(out["diam2"]), k, byref(n), int(on_device)))
        return out

    def filtration(self, cloud: int = 0) -> dict:
        n = c_int64(0)
        self._check(self.lib.ph_get_filtration(self._h, cloud, None, None, None, None, None,
                                               byref(n)))
        k = n.value
        out = dict(dim=np.empty(k, np.int32), diam2=np.empty(k, np.int64),
                   verts=np.empty((k, 6), np.int32), beta=np.empty(k, np.int32),
                   low=np.empty(k, np.int32))
        self._check(self.lib.ph_get_filtration(self._h, cloud, _ptr(out["dim"]),
                                               _ptr(out["diam2"]), _ptr(out["verts"]),
                                               _ptr(out["beta"]), _ptr(out["low"]), byref(n)))
        return out
