"""CPU oracle for the persistent-homology path of arXiv:1708.04710 -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import this package. The product library never loads it, and the two
share no code: the oracle is plain sequential C (``ph_oracle.c``) plus the numpy glue below.

Functions (indices are 0-based global filtration positions, -1 means "none"):

* ``vr_build``        Vietoris-Rips filtration and boundary matrix (Sec. 2.2-2.3).
* ``boundary_from_simplices``  boundary matrix of an explicit, compatibly ordered complex.
* ``beta``            beta of Definition 4 via Algorithm 4.
* ``reduce_std``      Algorithm 1 (optionally with V, R = D V).
* ``reduce_twist``    Algorithm 3 (clearing).
* ``reduce_pms``      Algorithm 2, pass by pass (Phase 0 / I / II, clearing, Cor. 10 zero case).
* ``pairs_and_essential``  the partition Pos / Neg / Ess of Sec. 2.3 from lowstar (Lemma 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "ph_oracle.c"
_LIB_PATH = _HERE / "libph_oracle.so"
_lib = None

PS_FIELDS = ("active", "new_pivots", "zero_final", "cor10", "cleared", "targets", "adds",
             "xors", "ess_est", "predicted", "empty_l")


def build_lib(force: bool = False) -> Path:
    """Compile the oracle with the host C compiler (no GPU involved)."""
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", str(_SRC), "-o",
                               str(tmp)])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build_lib()
        L = ctypes.CDLL(str(_LIB_PATH))
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        L.orc_vr_build.argtypes = [P, i32, i32, i32, i64, ctypes.POINTER(P)]
        L.orc_vr_build.restype = ctypes.c_int
        L.orc_vr_build_scales.argtypes = [P, i32, i32, i32, i64, i32, ctypes.POINTER(P)]
        L.orc_vr_build_scales.restype = ctypes.c_int
        L.orc_complex_size.argtypes = [P]
        L.orc_complex_size.restype = i64
        L.orc_complex_nnz.argtypes = [P]
        L.orc_complex_nnz.restype = i64
        L.orc_complex_export.argtypes = [P, P, P, P, P, P]
        L.orc_complex_export.restype = None
        L.orc_complex_free.argtypes = [P]
        L.orc_complex_free.restype = None
        L.orc_beta.argtypes = [i64, P, P, P]
        L.orc_beta.restype = ctypes.c_int
        L.orc_reduce_std.argtypes = [i64, P, P, P, P, P, P]
        L.orc_reduce_std.restype = ctypes.c_int
        L.orc_reduce_twist.argtypes = [i64, P, P, P, P, P]
        L.orc_reduce_twist.restype = ctypes.c_int
        L.orc_reduce_pms.argtypes = [i64, P, P, P, P, i32, i32, i32, i32, i32, P, P, P, P, P, P]
        L.orc_reduce_pms.restype = ctypes.c_int
        L.orc_reduce_pms_columns.argtypes = [i64, P, P, P, P, i32, i32, i32, i32, i32, P, P, P,
                                             i64, P]
        L.orc_reduce_pms_columns.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


class Complex(dict):
    """Filtration + boundary matrix: keys dim, diam2, verts (m x 4), colptr, rows."""

    @property
    def m(self) -> int:
        return int(self["dim"].shape[0])


VR_NV = 6  # vertex slots per simplex of a VR build (dimension <= 5), -1 padded


def vr_build(coords: np.ndarray, max_dim: int, max_diam2: int = -1, scale_step: int = 0,
             n_scales: int = 0) -> Complex:
    """Vietoris-Rips filtration of int32 grid points (Sec. 2.2) with its boundary matrix. With
    scale_step > 0 the filtration values are indices on the grid of scales r_i = i * scale_step
    (i = 0..n_scales, Sec. 4) and "diam2" holds them."""
    L = _load()
    c = np.ascontiguousarray(coords, dtype=np.int32)
    n, D = c.shape
    h = ctypes.c_void_p()
    if scale_step > 0:
        rc = L.orc_vr_build_scales(_ptr(c), n, D, max_dim, int(scale_step), int(n_scales),
                                   ctypes.byref(h))
    else:
        rc = L.orc_vr_build(_ptr(c), n, D, max_dim, int(max_diam2), ctypes.byref(h))
    if rc != 0:
        raise RuntimeError(f"orc_vr_build failed: {rc}")
    try:
        m = L.orc_complex_size(h)
        nnz = L.orc_complex_nnz(h)
        K = Complex(dim=np.empty(m, np.int32), diam2=np.empty(m, np.int64),
                    verts=np.empty((m, VR_NV), np.int32), colptr=np.empty(m + 1, np.int64),
                    rows=np.empty(max(nnz, 1), np.int32))
        L.orc_complex_export(h, _ptr(K["dim"]), _ptr(K["diam2"]), _ptr(K["verts"]),
                             _ptr(K["colptr"]), _ptr(K["rows"]))
        K["rows"] = K["rows"][:nnz]
    finally:
        L.orc_complex_free(h)
    return K


def boundary_from_simplices(simplices) -> Complex:
    """Boundary matrix (Eq. def:boundary_matrix) of an explicit complex given as a list of
    vertex tuples in a compatible order (every face listed before its cofaces)."""
    index = {}
    dims, colptr, rows = [], [0], []
    verts = np.full((len(simplices), 4), -1, np.int32)
    for j, s in enumerate(simplices):
        s = tuple(sorted(s))
        index[s] = j
        d = len(s) - 1
        dims.append(d)
        if len(s) <= 4:
            verts[j, :len(s)] = s
        if d > 0:
            faces = sorted(index[s[:k] + s[k + 1:]] for k in range(len(s)))
            rows.extend(faces)
        colptr.append(len(rows))
    return Complex(dim=np.array(dims, np.int32), diam2=np.zeros(len(simplices), np.int64),
                   verts=verts, colptr=np.array(colptr, np.int64),
                   rows=np.array(rows, np.int32))


def beta(K: Complex) -> np.ndarray:
    L = _load()
    out = np.empty(K.m, np.int32)
    rc = L.orc_beta(K.m, _ptr(K["colptr"]), _ptr(K["rows"]), _ptr(out))
    if rc != 0:
        raise RuntimeError(rc)
    return out


def reduce_std(K: Complex, track_v: bool = False):
    """Algorithm 1. Returns (low, stats[adds, xors]) or, with track_v, (low, stats, R, V)."""
    L = _load()
    m = K.m
    low = np.empty(m, np.int32)
    st = np.zeros(2, np.int64)
    R = V = None
    if track_v:
        R = np.zeros((m, m), np.uint8)
        V = np.zeros((m, m), np.uint8)
    rc = L.orc_reduce_std(m, _ptr(K["colptr"]), _ptr(K["rows"]), _ptr(low), _ptr(st),
                          _ptr(R) if track_v else None, _ptr(V) if track_v else None)
    if rc != 0:
        raise RuntimeError(rc)
    return (low, st, R, V) if track_v else (low, st)


def reduce_twist(K: Complex):
    """Algorithm 3. Returns (low, stats[adds, xors, cleared])."""
    L = _load()
    low = np.empty(K.m, np.int32)
    st = np.zeros(3, np.int64)
    rc = L.orc_reduce_twist(K.m, _ptr(K["colptr"]), _ptr(K["rows"]), _ptr(K["dim"]), _ptr(low),
                            _ptr(st))
    if rc != 0:
        raise RuntimeError(rc)
    return low, st


class PmsResult(dict):
    """low, passes, stats (rows per executed pass, columns PS_FIELDS), ess_est, proven,
    predicted (Corollary 10 non-zero case: lowstar of the column, or -1), converged."""

    def __getattr__(self, k):
        return self[k]


def reduce_pms(K: Complex, max_passes: int = 100000, strict: bool = False, cor10: bool = True,
               beta_arr: np.ndarray | None = None, sets: int = 0,
               priority: int = 0) -> PmsResult:
    """Algorithm 2, pass by pass (see ph_oracle.c for the pass definition). sets > 0: Phase II
    acts on that many neighbour sets per pass, ordered by |N| (priority 0) or by known-negative
    targets first (priority 1), Sec. 3.4."""
    L = _load()
    m = K.m
    b = beta(K) if beta_arr is None else np.ascontiguousarray(beta_arr, np.int32)
    low = np.empty(m, np.int32)
    ps = np.zeros((max_passes + 1, len(PS_FIELDS)), np.int64)
    npass = ctypes.c_int32(0)
    ess = np.zeros(max(m, 1), np.uint8)
    proven = np.zeros(max(m, 1), np.uint8)
    pred = np.full(max(m, 1), -1, np.int32)
    rc = L.orc_reduce_pms(m, _ptr(K["colptr"]), _ptr(K["rows"]), _ptr(K["dim"]), _ptr(b),
                          max_passes, int(strict), int(cor10), int(sets), int(priority),
                          _ptr(low), _ptr(ps),
                          ctypes.byref(npass), _ptr(ess), _ptr(proven), _ptr(pred))
    if rc < 0:
        raise RuntimeError(rc)
    p = npass.value
    return PmsResult(low=low, passes=p, stats=ps[:p + 1], ess_est=ess[:m].astype(bool),
                     proven=proven[:m].astype(bool), predicted=pred[:m], converged=(rc == 0))


def reduce_pms_columns(K: Complex, max_passes: int = 100000, strict: bool = False,
                       cor10: bool = True, sets: int = 0, priority: int = 0):
    """The reduced matrix R that Algorithm 2 (as reduce_pms) leaves: (colptr int64 [m + 1],
    rows int32 [nnz]), CSC with ascending rows."""
    L = _load()
    m = K.m
    b = beta(K)
    low = np.empty(max(m, 1), np.int32)
    cp = np.zeros(m + 1, np.int64)
    nnz = ctypes.c_int64(0)
    args = (m, _ptr(K["colptr"]), _ptr(K["rows"]), _ptr(K["dim"]), _ptr(b), max_passes,
            int(strict), int(cor10), int(sets), int(priority), _ptr(low), _ptr(cp))
    rc = L.orc_reduce_pms_columns(*args, None, 0, ctypes.byref(nnz))
    if rc < 0:
        raise RuntimeError(rc)
    rows = np.zeros(max(nnz.value, 1), np.int32)
    rc = L.orc_reduce_pms_columns(*args, _ptr(rows), nnz.value, ctypes.byref(nnz))
    if rc < 0:
        raise RuntimeError(rc)
    return cp, rows[:nnz.value]


def pairs_and_essential(low: np.ndarray, dim: np.ndarray):
    """Pairs (lowstar(j), j) of negative columns and the essential set (Sec. 2.3, Lemma 1).

    Returns (pairs int64 (P, 2) sorted by death index, essential int64 sorted)."""
    low = np.asarray(low, np.int64)
    deaths = np.nonzero(low >= 0)[0]
    births = low[deaths]
    pairs = np.stack([births, deaths], axis=1) if deaths.size else np.zeros((0, 2), np.int64)
    paired = np.zeros(low.shape[0], bool)
    paired[deaths] = True
    paired[births] = True
    essential = np.nonzero(~paired)[0].astype(np.int64)
    return pairs.astype(np.int64), essential


def persistence_summary(K: Complex, low: np.ndarray):
    """Per dimension: (#finite pairs by birth dim, #essential by dim)."""
    pairs, ess = pairs_and_essential(low, K["dim"])
    maxd = int(K["dim"].max()) if K.m else 0
    npairs = np.bincount(K["dim"][pairs[:, 0]], minlength=maxd + 1) if len(pairs) else np.zeros(
        maxd + 1, np.int64)
    ness = np.bincount(K["dim"][ess], minlength=maxd + 1)
    return npairs, ness


# ----------------------------------------------------------------------------------------------
# Differentiable diagram loss (FP64 reference). The pairing comes from lowstar; the birth and
# death values of a pair are Euclidean diameters (Sec. 2.2); a simplex's diameter is realised by
# an edge: an edge by itself, a higher simplex by the realising edge of its last face in the
# filtration (the largest row of its boundary column).
# ----------------------------------------------------------------------------------------------
def realising_edge(K: Complex, x: int):
    while K["dim"][x] > 1:
        x = int(K["rows"][K["colptr"][x + 1] - 1])
    return int(K["verts"][x, 0]), int(K["verts"][x, 1])


def diagram_edges(K: Complex, low: np.ndarray, dim: int) -> np.ndarray:
    """(p, q, r, s) per finite pair whose birth simplex has dimension `dim`: birth realised by
    edge (p, q) (-1, -1 for a vertex birth), death by edge (r, s)."""
    out = []
    for j in np.nonzero((np.asarray(low) >= 0) & (K["dim"] == dim + 1))[0]:
        r, s = realising_edge(K, int(j))
        b = int(low[j])
        p, q = realising_edge(K, b) if K["dim"][b] >= 1 else (-1, -1)
        out.append((p, q, r, s))
    return np.array(out, np.int64).reshape(-1, 4)


def diagram_loss_grad(x: np.ndarray, edges: np.ndarray):
    """loss = sum over pairs (d - b)^2 with b = |x_p - x_q|, d = |x_r - x_s| (float64), and its
    gradient with respect to x; zero-length edges contribute no gradient."""
    x = np.asarray(x, np.float64)
    grad = np.zeros_like(x)
    loss = 0.0
    for p, q, r, s in edges:
        dv = x[r] - x[s]
        d = float(np.sqrt(dv @ dv))
        if p >= 0:
            bv = x[p] - x[q]
            b = float(np.sqrt(bv @ bv))
        else:
            bv, b = None, 0.0
        loss += (d - b) ** 2
        g = 2.0 * (d - b)
        if d > 0:
            grad[r] += g * dv / d
            grad[s] -= g * dv / d
        if p >= 0 and b > 0:
            grad[p] -= g * bv / b
            grad[q] += g * bv / b
    return loss, grad
