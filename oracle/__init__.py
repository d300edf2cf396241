"""CPU oracle for the Slim Graph hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product path (the CUDA
library and its binding) never loads it and never falls back to it.

The arithmetic lives in ``sg_oracle.c`` (plain single-threaded C, FP64 for
floating point), compiled with gcc into ``liboracle.so`` beside this file on
first use.  This module only marshals numpy arrays in and out of it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

UNIFORM, SPECTRAL_LOGN, SPECTRAL_AVGDEG, TR_RANDOM, TR_MAXW, TR_EO, TR_EO_MAXW, TR_P2, TR_MINCOUNT, \
    TR_EO_MINCOUNT = range(10)
KERNELS = {
    "uniform": UNIFORM, "spectral_logn": SPECTRAL_LOGN, "spectral_avgdeg": SPECTRAL_AVGDEG,
    "tr_random": TR_RANDOM, "tr_maxw": TR_MAXW, "tr_eo": TR_EO, "tr_eo_maxw": TR_EO_MAXW,
    "tr_p2": TR_P2, "tr_mincount": TR_MINCOUNT, "tr_eo_mincount": TR_EO_MINCOUNT,
}


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no GPU, no CUDA involved)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB)
    i64, u64, dbl, vp = C.c_int64, C.c_uint64, C.c_double, C.c_void_p
    lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
    lib.orc_philox4x32_10.restype = None
    lib.orc_threshold.argtypes = [dbl]
    lib.orc_threshold.restype = u64
    lib.orc_triangle_count.argtypes = [i64, vp, vp]
    lib.orc_triangle_count.restype = i64
    lib.orc_triangle_list.argtypes = [i64, vp, vp, vp, i64]
    lib.orc_triangle_list.restype = i64
    lib.orc_compress.argtypes = [i64, i64, vp, vp, vp, C.c_int, dbl, u64, C.c_int, vp, vp, vp, vp]
    lib.orc_compress.restype = i64
    lib.orc_tr_union_edge_deleted.argtypes = [i64, vp, vp, vp, C.c_int, dbl, u64, C.c_uint32, C.c_uint32]
    lib.orc_tr_union_edge_deleted.restype = C.c_int
    lib.orc_pagerank.argtypes = [i64, vp, vp, dbl, C.c_int, vp]
    lib.orc_pagerank.restype = dbl
    lib.orc_kl_divergence.argtypes = [i64, vp, vp]
    lib.orc_kl_divergence.restype = dbl
    lib.orc_cc_count.argtypes = [i64, vp, vp, vp]
    lib.orc_cc_count.restype = i64
    lib.orc_mst_weight_units.argtypes = [i64, vp, vp, vp]
    lib.orc_mst_weight_units.restype = i64
    lib.orc_low_degree.argtypes = [i64, vp, vp, vp, vp, vp, vp]
    lib.orc_low_degree.restype = i64
    lib.orc_bfs_levels.argtypes = [i64, vp, vp, i64, vp]
    lib.orc_bfs_levels.restype = None
    lib.orc_critical_edges.argtypes = [i64, vp, vp, i64]
    lib.orc_critical_edges.restype = i64
    lib.orc_reordered_neighbours.argtypes = [i64, vp, vp, vp, vp]
    lib.orc_reordered_neighbours.restype = i64
    lib.orc_vertex_triangle_counts.argtypes = [i64, vp, vp, vp]
    lib.orc_vertex_triangle_counts.restype = None
    lib.orc_reordered_neighbours_i64.argtypes = [i64, vp, vp, vp, vp]
    lib.orc_reordered_neighbours_i64.restype = i64
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data


def _arrays(g):
    """Accept a graphgen.CSR or an (n, off, col, w) tuple; return numpy arrays."""
    if isinstance(g, tuple):
        n, off, col, w = g
    else:
        n = g.n
        off, col, w = g.numpy()
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col).view(np.uint32) if col.dtype != np.uint32 else np.ascontiguousarray(col)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    return int(n), off, col, w


def philox4x32_10(ctr, key):
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def threshold(p: float) -> int:
    return int(_load().orc_threshold(float(p)))


def triangle_count(g) -> int:
    n, off, col, _ = _arrays(g)
    return int(_load().orc_triangle_count(n, _p(off), _p(col)))


def triangle_list(g) -> np.ndarray:
    n, off, col, _ = _arrays(g)
    lib = _load()
    t = int(lib.orc_triangle_count(n, _p(off), _p(col)))
    out = np.zeros((max(t, 1), 3), dtype=np.uint32)
    lib.orc_triangle_list(n, _p(off), _p(col), _p(out), t)
    return out[:t]


class OracleError(RuntimeError):
    pass


def compress(g, kernel, p: float, seed: int, want_weights: bool = False, return_accepted: bool = False):
    """compress(G, kernel, p, seed) -> (off', col', w' or None[, accepted-arc mask])."""
    n, off, col, w = _arrays(g)
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    nnz = int(col.size)
    off_o = np.zeros(n + 1, dtype=np.int64)
    col_o = np.zeros(max(nnz, 1), dtype=np.uint32)
    spectral = k in (SPECTRAL_LOGN, SPECTRAL_AVGDEG)
    has_w = (w is not None) or (spectral and want_weights)
    w_o = np.zeros(max(nnz, 1), dtype=np.float32) if has_w else None
    acc = np.zeros(max(nnz, 1), dtype=np.uint8) if return_accepted else None
    r = int(_load().orc_compress(n, nnz, _p(off), _p(col), _p(w), k, float(p), int(seed) & (2**64 - 1),
                                 int(bool(want_weights)), _p(off_o), _p(col_o), _p(w_o), _p(acc)))
    if r < 0:
        raise OracleError({-1: "invalid argument", -2: "kernel needs weights", -3: "out of memory"}[r])
    res = (off_o, col_o[:r].copy(), None if w_o is None else w_o[:r].copy())
    if return_accepted:
        return res + (acc[:nnz].copy(),)
    return res


def tr_union_edge_deleted(g, kernel, p: float, seed: int, x: int, y: int) -> bool:
    n, off, col, w = _arrays(g)
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    return bool(_load().orc_tr_union_edge_deleted(n, _p(off), _p(col), _p(w), k, float(p),
                                                  int(seed) & (2**64 - 1), int(x), int(y)))


def pagerank(g, damping: float = 0.85, iters: int = 50):
    """FP64 PageRank vector and the final L1 residual."""
    n, off, col, _ = _arrays(g)
    x = np.zeros(max(n, 1), dtype=np.float64)
    r = float(_load().orc_pagerank(n, _p(off), _p(col), float(damping), int(iters), _p(x)))
    return x[:n], r


def kl_divergence(P, Q) -> float:
    P = np.ascontiguousarray(P, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    assert P.shape == Q.shape
    return float(_load().orc_kl_divergence(P.size, _p(P), _p(Q)))


def cc_count(g, return_labels: bool = False):
    n, off, col, _ = _arrays(g)
    lab = np.zeros(max(n, 1), dtype=np.int64) if return_labels else None
    c = int(_load().orc_cc_count(n, _p(off), _p(col), _p(lab)))
    return (c, lab[:n]) if return_labels else c


def mst_weight_units(g) -> int:
    n, off, col, w = _arrays(g)
    if w is None:
        raise OracleError("mst needs weights")
    return int(_load().orc_mst_weight_units(n, _p(off), _p(col), _p(w)))


def divergence(g, h, damping: float = 0.85, iters: int = 50):
    """The accuracy analytics of one compression: KL(PR_G || PR_H) and #CC."""
    P, rg = pagerank(g, damping, iters)
    Q, rh = pagerank(h, damping, iters)
    return {"kl_bits": kl_divergence(P, Q), "cc_g": cc_count(g), "cc_h": cc_count(h),
            "pr_residual_g": rg, "pr_residual_h": rh}


def low_degree(g):
    """low_degree (Listing 1): drop every vertex of degree 0 or 1.
    Returns (n', off', col', new_id) with new_id[v] = -1 for dropped vertices."""
    n, off, col, _ = _arrays(g)
    new_id = np.zeros(max(n, 1), dtype=np.int64)
    off_o = np.zeros(n + 1, dtype=np.int64)
    col_o = np.zeros(max(col.size, 1), dtype=np.uint32)
    nnz = C.c_int64()
    k = int(_load().orc_low_degree(n, _p(off), _p(col), _p(new_id), _p(off_o), _p(col_o), C.addressof(nnz)))
    return k, off_o[:k + 1].copy(), col_o[:nnz.value].copy(), new_id[:n].copy()


def bfs_levels(g, root: int) -> np.ndarray:
    n, off, col, _ = _arrays(g)
    lev = np.zeros(max(n, 1), dtype=np.int64)
    _load().orc_bfs_levels(n, _p(off), _p(col), int(root), _p(lev))
    return lev[:n]


def critical_edges(g, root: int) -> int:
    """|E_cr| of a BFS from root: edges joining consecutive levels (Sec. 5.3)."""
    n, off, col, _ = _arrays(g)
    return int(_load().orc_critical_edges(n, _p(off), _p(col), int(root)))


def reordered_neighbours(g, x, y) -> int:
    """Edges of g whose endpoint order under score x differs from that under y (A_REN count).
    Float32 scores are compared in float32; int64 scores exactly."""
    n, off, col, _ = _arrays(g)
    if np.asarray(x).dtype.kind in "iu":
        x = np.ascontiguousarray(x, dtype=np.int64)
        y = np.ascontiguousarray(y, dtype=np.int64)
        assert x.size == n and y.size == n
        return int(_load().orc_reordered_neighbours_i64(n, _p(off), _p(col), _p(x), _p(y)))
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    assert x.size == n and y.size == n
    return int(_load().orc_reordered_neighbours(n, _p(off), _p(col), _p(x), _p(y)))


def vertex_triangle_counts(g) -> np.ndarray:
    """Triangles through every vertex."""
    n, off, col, _ = _arrays(g)
    out = np.zeros(max(n, 1), dtype=np.int64)
    _load().orc_vertex_triangle_counts(n, _p(off), _p(col), _p(out))
    return out[:n]
