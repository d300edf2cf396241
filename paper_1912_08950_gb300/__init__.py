"""Slim Graph lossy graph compression on one GB300 (sm_103a).

A thin ctypes binding over ``libslimgraph.so`` (declared in
``include/slimgraph.h``).  Every step of compression and analytics runs in the
library's CUDA kernels; this module only marshals arguments.  PyTorch is used
for device memory and streams.  There is no CPU fallback: if the library has
not been built, importing this package raises ImportError.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libslimgraph.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = C.CDLL(LIB_PATH)

SG_OK, SG_ERR_INVALID_ARG, SG_ERR_INVALID_GRAPH, SG_ERR_NEEDS_WEIGHTS, SG_ERR_OOM, SG_ERR_CUDA, \
    SG_ERR_TIMEOUT, SG_ERR_UNSUPPORTED = range(8)
STATUS_NAMES = {0: "SG_OK", 1: "SG_ERR_INVALID_ARG", 2: "SG_ERR_INVALID_GRAPH", 3: "SG_ERR_NEEDS_WEIGHTS",
                4: "SG_ERR_OOM", 5: "SG_ERR_CUDA", 6: "SG_ERR_TIMEOUT", 7: "SG_ERR_UNSUPPORTED"}

KERNELS = {"uniform": 0, "spectral_logn": 1, "spectral_avgdeg": 2, "tr_random": 3, "tr_maxw": 4,
           "tr_eo": 5, "tr_eo_maxw": 6, "tr_p2": 7, "tr_mincount": 8, "tr_eo_mincount": 9}


class SgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class CsrView(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("off", C.c_void_p), ("col", C.c_void_p),
                ("w", C.c_void_p)]


class DivResult(C.Structure):
    _fields_ = [("kl_bits", C.c_double), ("cc_g", C.c_int64), ("cc_h", C.c_int64), ("m_g", C.c_int64),
                ("m_h", C.c_int64), ("pr_residual_g", C.c_double), ("pr_residual_h", C.c_double)]


class AccuracyResult(C.Structure):
    _fields_ = [("m_g", C.c_int64), ("pr_reordered", C.c_int64), ("pr_aren", C.c_double),
                ("tc_reordered", C.c_int64), ("tc_aren", C.c_double), ("root", C.c_int64),
                ("critical_g", C.c_int64), ("critical_h", C.c_int64), ("critical_fraction", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_uint64), ("probes", C.c_uint64), ("triangles", C.c_uint64),
                ("eo_rounds", C.c_uint64), ("eo_listed", C.c_uint64), ("eo_passes", C.c_uint64),
                ("eo_list_passes", C.c_uint64)]


_vp, _i64, _u64, _int, _dbl, _flt = C.c_void_p, C.c_int64, C.c_uint64, C.c_int, C.c_double, C.c_float
_PP = C.POINTER(C.c_void_p)
_SIGS = {
    "sg_ctx_create": [_int, _vp, _PP],
    "sg_ctx_synchronize": [_vp],
    "sg_ctx_stats": [_vp, C.POINTER(Stats), _int],
    "sg_ctx_set_profiling": [_vp, _int],
    "sg_ctx_kernel_time": [_vp, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)],
    "sg_ctx_reset_profile": [_vp],
    "sg_ctx_set_eo_list_capacity": [_vp, _i64],
    "sg_ctx_release_workspace": [_vp],
    "sg_device_free_memory": [_int, C.POINTER(C.c_uint64)],
    "sg_ctx_set_scan_hold": [_vp, C.c_uint32],
    "sg_kernel_arch": [_int, C.POINTER(C.c_int)],
    "sg_graph_from_device": [_vp, C.POINTER(CsrView), _int, _int, _PP],
    "sg_graph_from_host": [_vp, _i64, _i64, _vp, _vp, _vp, _PP],
    "sg_graph_view": [_vp, C.POINTER(CsrView)],
    "sg_graph_download": [_vp, _vp, _vp, _vp, _vp],
    "sg_compress": [_vp, _vp, _int, _dbl, _u64, _int, _PP],
    "sg_divergence": [_vp, _vp, _vp, _flt, _int, C.POINTER(DivResult)],
    "sg_pagerank": [_vp, _vp, _flt, _int, _vp, C.POINTER(C.c_double)],
    "sg_kl_divergence": [_vp, _i64, _vp, _vp, C.POINTER(C.c_double)],
    "sg_cc_count": [_vp, _vp, C.POINTER(C.c_int64), _vp],
    "sg_triangle_count": [_vp, _vp, C.POINTER(C.c_int64)],
    "sg_compress_uniform_noalloc": [_int, _vp, _i64, _i64, _vp, _vp, _dbl, _u64, _vp, _vp, C.POINTER(C.c_int64)],
    "sg_batch_create": [_vp, _int, C.POINTER(C.c_void_p), _PP],
    "sg_compress_batch": [_vp, _vp, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_uint64), _int,
                          C.POINTER(C.c_void_p)],
    "sg_batch_info": [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int),
                      C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "sg_tr_work": [_vp, _vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                   C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "sg_low_degree": [_vp, _vp, _vp, _PP],
    "sg_bfs_levels": [_vp, _vp, _i64, _vp],
    "sg_critical_edges": [_vp, _vp, _i64, C.POINTER(C.c_int64)],
    "sg_reordered_neighbours": [_vp, _vp, _vp, _vp, C.POINTER(C.c_int64)],
    "sg_vertex_triangle_counts": [_vp, _vp, _vp],
    "sg_accuracy": [_vp, _vp, _vp, _flt, _int, _i64, C.POINTER(AccuracyResult)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _int
_lib.sg_ctx_destroy.argtypes = [_vp]
_lib.sg_ctx_destroy.restype = None
_lib.sg_batch_free.argtypes = [_vp]
_lib.sg_batch_free.restype = None
_lib.sg_graph_free.argtypes = [_vp]
_lib.sg_graph_free.restype = None
_lib.sg_last_error.argtypes = []
_lib.sg_last_error.restype = C.c_char_p


def lib():
    """The loaded ctypes library (for callers that want the raw C-ABI)."""
    return _lib


def _check(st: int):
    if st != SG_OK:
        raise SgError(st, (_lib.sg_last_error() or b"").decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


class Context:
    """A device, a stream and the library's per-context state."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        self.device = device
        if stream is None:
            stream = torch.cuda.Stream(device)
        self.torch_stream = stream
        h = C.c_void_p()
        _check(_lib.sg_ctx_create(device, C.c_void_p(stream.cuda_stream), C.byref(h)))
        self.handle = h
        self._graphs = weakref.WeakSet()
        self._batches = weakref.WeakSet()

    def close(self):
        """Free every graph and batch still alive on this context, then the context."""
        if getattr(self, "handle", None):
            for b in list(self._batches):
                b.free()
            for g in list(self._graphs):
                g.free()
            _lib.sg_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def synchronize(self):
        _check(_lib.sg_ctx_synchronize(self.handle))

    def stats(self, reset: bool = False) -> dict:
        s = Stats()
        _check(_lib.sg_ctx_stats(self.handle, C.byref(s), int(reset)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def set_profiling(self, on: bool):
        _check(_lib.sg_ctx_set_profiling(self.handle, int(on)))

    def kernel_time(self, prefix: str):
        ms, n = C.c_double(), C.c_int64()
        _check(_lib.sg_ctx_kernel_time(self.handle, prefix.encode(), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def reset_profile(self):
        _check(_lib.sg_ctx_reset_profile(self.handle))

    def set_eo_list_capacity(self, records: int):
        """0: automatic, -1: no triangle list, > 0: at most that many triangles."""
        _check(_lib.sg_ctx_set_eo_list_capacity(self.handle, int(records)))

    def set_scan_hold(self, spin_limit: int):
        """Test hook: make every prefix scan's first wait run out (0: off)."""
        _check(_lib.sg_ctx_set_scan_hold(self.handle, int(spin_limit)))

    def release_workspace(self):
        """Free the edge-once list workspaces the context keeps between calls."""
        _check(_lib.sg_ctx_release_workspace(self.handle))


class Graph:
    """A device-resident symmetric CSR owned (or borrowed) by the library."""

    def __init__(self, ctx: Context, handle, keepalive=None):
        self.ctx = ctx
        self.handle = handle
        self._keep = keepalive
        ctx._graphs.add(self)
        v = CsrView()
        _check(_lib.sg_graph_view(self.handle, C.byref(v)))
        self.n, self.nnz = v.n, v.nnz
        self.weighted = bool(v.w)

    @property
    def m(self) -> int:
        return self.nnz // 2

    @classmethod
    def from_host(cls, ctx: Context, n: int, off: np.ndarray, col: np.ndarray, w: Optional[np.ndarray] = None):
        off = np.ascontiguousarray(off, dtype=np.int64)
        col = np.ascontiguousarray(col).view(np.uint32)
        w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
        h = C.c_void_p()
        _check(_lib.sg_graph_from_host(ctx.handle, n, col.size, _ptr(off), _ptr(col), _ptr(w), C.byref(h)))
        return cls(ctx, h)

    @classmethod
    def from_tensors(cls, ctx: Context, n: int, off, col, w=None, copy: bool = False, validate: bool = False):
        """Wrap (copy=False) or copy CUDA tensors: off int64[n+1], col int32/uint32[nnz], w float32[nnz]."""
        import torch

        # the tensors may still be in flight on the producer's stream
        ctx.torch_stream.wait_stream(torch.cuda.current_stream(ctx.device))
        v = CsrView(n, col.numel(), off.data_ptr(), col.data_ptr(), None if w is None else w.data_ptr())
        h = C.c_void_p()
        _check(_lib.sg_graph_from_device(ctx.handle, C.byref(v), int(copy), int(validate), C.byref(h)))
        return cls(ctx, h, keepalive=None if copy else (off, col, w))

    @classmethod
    def from_csr(cls, ctx: Context, g, copy: bool = True, validate: bool = False):
        """From a graphgen.CSR (on any device)."""
        import torch

        dev = torch.device("cuda", ctx.device)
        off, col = g.off.to(dev).contiguous(), g.col.to(dev).contiguous()
        w = None if g.w is None else g.w.to(dev).contiguous()
        return cls.from_tensors(ctx, g.n, off, col, w, copy=copy, validate=validate)

    def tensors(self):
        """Zero-copy CUDA tensors (off int64, col int32, w float32 or None) over the
        graph's device arrays; valid only while this graph is alive."""
        import torch

        v = CsrView()
        _check(_lib.sg_graph_view(self.handle, C.byref(v)))

        class _Arr:
            def __init__(self, ptr, n, typestr):
                self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr or 0, False),
                                                 "version": 3, "strides": None}

        dev = torch.device("cuda", self.ctx.device)
        off = torch.as_tensor(_Arr(v.off, v.n + 1, "<i8"), device=dev)
        col = torch.as_tensor(_Arr(v.col, v.nnz, "<i4"), device=dev) if v.nnz else torch.zeros(0, dtype=torch.int32, device=dev)
        w = torch.as_tensor(_Arr(v.w, v.nnz, "<f4"), device=dev) if (v.w and v.nnz) else None
        return off, col, w

    def download(self):
        off = np.zeros(self.n + 1, dtype=np.int64)
        col = np.zeros(max(self.nnz, 1), dtype=np.uint32)
        w = np.zeros(max(self.nnz, 1), dtype=np.float32) if self.weighted else None
        _check(_lib.sg_graph_download(self.ctx.handle, self.handle, _ptr(off), _ptr(col), _ptr(w)))
        return off, col[:self.nnz], (None if w is None else w[:self.nnz])

    def free(self):
        if getattr(self, "handle", None):
            _lib.sg_graph_free(self.handle)
            self.handle = None
            self._keep = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def device_free_memory(device: int = 0) -> int:
    """Bytes of device memory free for new work (driver free + unused pool memory)."""
    v = C.c_uint64()
    _check(_lib.sg_device_free_memory(int(device), C.byref(v)))
    return v.value


def compress(g: Graph, kernel, p: float, seed: int, want_weights: bool = False) -> Graph:
    """compress(G, kernel, p, seed) -> H (Listing 1 kernels; see slimgraph.h)."""
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    h = C.c_void_p()
    _check(_lib.sg_compress(g.ctx.handle, g.handle, k, float(p), int(seed) & (2**64 - 1), int(want_weights),
                            C.byref(h)))
    return Graph(g.ctx, h)


def low_degree(g: Graph, return_map: bool = False):
    """low_degree(V v) (Listing 1): H = G without its vertices of degree 0 or 1,
    renumbered in id order.  With return_map, also the device uint32 tensor
    mapping H's vertex ids to G's."""
    import torch

    nto = torch.empty(max(g.n, 1), dtype=torch.int32, device=f"cuda:{g.ctx.device}") if return_map else None
    if nto is not None:
        torch.cuda.current_stream(g.ctx.device).synchronize()
    h = C.c_void_p()
    _check(_lib.sg_low_degree(g.ctx.handle, g.handle, None if nto is None else nto.data_ptr(), C.byref(h)))
    H = Graph(g.ctx, h)
    if nto is None:
        return H
    g.ctx.synchronize()
    return H, nto[:H.n]


def divergence(g: Graph, h: Graph, damping: float = 0.85, iters: int = 50) -> dict:
    r = DivResult()
    _check(_lib.sg_divergence(g.ctx.handle, g.handle, h.handle, float(damping), int(iters), C.byref(r)))
    return {k: getattr(r, k) for k, _ in DivResult._fields_}


def pagerank(g: Graph, damping: float = 0.85, iters: int = 50):
    """FP32 PageRank vector (a CUDA tensor) and the FP64 residual of the last update."""
    import torch

    x = torch.empty(max(g.n, 1), dtype=torch.float32, device=torch.device("cuda", g.ctx.device))
    r = C.c_double()
    _check(_lib.sg_pagerank(g.ctx.handle, g.handle, float(damping), int(iters), x.data_ptr(), C.byref(r)))
    return x[:g.n], r.value


def _dev_tensor(g: Graph, n: int, dtype):
    import torch

    t = torch.empty(max(n, 1), dtype=dtype, device=torch.device("cuda", g.ctx.device))
    g.ctx.torch_stream.wait_stream(torch.cuda.current_stream(g.ctx.device))
    return t


def _publish(ctx: Context):
    import torch

    torch.cuda.current_stream(ctx.device).wait_stream(ctx.torch_stream)


def bfs_levels(g: Graph, root: int):
    """Hop distance of every vertex from root (int32 CUDA tensor, -1 = unreached; Sec. 5.3)."""
    import torch

    lev = _dev_tensor(g, g.n, torch.int32)
    _check(_lib.sg_bfs_levels(g.ctx.handle, g.handle, int(root), lev.data_ptr()))
    _publish(g.ctx)
    return lev[:g.n]


def critical_edges(g: Graph, root: int) -> int:
    """|E_cr| of a BFS from root: the edges joining consecutive levels (Sec. 5.3)."""
    out = C.c_int64()
    _check(_lib.sg_critical_edges(g.ctx.handle, g.handle, int(root), C.byref(out)))
    return out.value


def reordered_neighbours(g: Graph, x, y) -> int:
    """Edges of g whose endpoint order under the float32 CUDA score x differs under y (A_REN count)."""
    import torch

    assert x.dtype == torch.float32 and y.dtype == torch.float32 and x.numel() == g.n and y.numel() == g.n
    x, y = x.contiguous(), y.contiguous()
    g.ctx.torch_stream.wait_stream(torch.cuda.current_stream(g.ctx.device))
    out = C.c_int64()
    _check(_lib.sg_reordered_neighbours(g.ctx.handle, g.handle, x.data_ptr(), y.data_ptr(), C.byref(out)))
    return out.value


def vertex_triangle_counts(g: Graph):
    """Triangles through every vertex (int64 CUDA tensor holding the uint64 counts)."""
    import torch

    t = _dev_tensor(g, g.n, torch.int64)
    _check(_lib.sg_vertex_triangle_counts(g.ctx.handle, g.handle, t.data_ptr()))
    _publish(g.ctx)
    return t[:g.n]


def accuracy(g: Graph, h: Graph, damping: float = 0.85, iters: int = 50, root: int = -1) -> dict:
    """A_REN of PageRank and of per-vertex triangle counts, and the BFS critical-edge fraction (Sec. 5)."""
    r = AccuracyResult()
    _check(_lib.sg_accuracy(g.ctx.handle, g.handle, h.handle, float(damping), int(iters), int(root), C.byref(r)))
    return {k: getattr(r, k) for k, _ in AccuracyResult._fields_}


def kl_divergence(ctx: Context, P, Q) -> float:
    import torch

    ctx.torch_stream.wait_stream(torch.cuda.current_stream(ctx.device))
    out = C.c_double()
    _check(_lib.sg_kl_divergence(ctx.handle, P.numel(), P.data_ptr(), Q.data_ptr(), C.byref(out)))
    return out.value


def cc_count(g: Graph, labels: bool = False):
    import torch

    cnt = C.c_int64()
    lab = torch.empty(max(g.n, 1), dtype=torch.int32, device=torch.device("cuda", g.ctx.device)) if labels else None
    _check(_lib.sg_cc_count(g.ctx.handle, g.handle, C.byref(cnt), None if lab is None else lab.data_ptr()))
    return (cnt.value, lab[:g.n]) if labels else cnt.value


def triangle_count(g: Graph) -> int:
    t = C.c_int64()
    _check(_lib.sg_triangle_count(g.ctx.handle, g.handle, C.byref(t)))
    return t.value


def tr_work(g: Graph) -> dict:
    m, w, md, t, ha, wf = (C.c_int64() for _ in range(6))
    _check(_lib.sg_tr_work(g.ctx.handle, g.handle, C.byref(m), C.byref(w), C.byref(md), C.byref(t), C.byref(ha),
                           C.byref(wf)))
    return {"m": m.value, "probes": w.value, "max_out_degree": md.value, "triangles": t.value,
            "head_arcs": ha.value, "forward_probes": wf.value}


class Batch:
    """Many graphs packed into one device-resident union (sg_batch_create)."""

    def __init__(self, ctx: Context, graphs):
        self.ctx = ctx
        self.count = len(graphs)
        arr = (C.c_void_p * self.count)(*[g.handle.value if hasattr(g.handle, "value") else g.handle
                                          for g in graphs])
        h = C.c_void_p()
        _check(_lib.sg_batch_create(ctx.handle, self.count, arr, C.byref(h)))
        self.handle = h
        self._outs = []
        ctx._batches.add(self)

    def compress(self, kernels, ps, seeds, want_weights: bool = False):
        """Compress every graph with its own kernel, p and seed (one CUDA-graph replay).
        The returned graphs are views valid until the next call or free()."""
        import torch

        self._release()
        self.ctx.torch_stream.wait_stream(torch.cuda.current_stream(self.ctx.device))
        ks = (C.c_int * self.count)(*[KERNELS[k] if isinstance(k, str) else int(k) for k in kernels])
        pv = (C.c_double * self.count)(*[float(p) for p in ps])
        sv = (C.c_uint64 * self.count)(*[int(x) & (2**64 - 1) for x in seeds])
        outs = (C.c_void_p * self.count)()
        _check(_lib.sg_compress_batch(self.ctx.handle, self.handle, ks, pv, sv, int(want_weights), outs))
        self._outs = [Graph(self.ctx, C.c_void_p(outs[i])) for i in range(self.count)]
        return list(self._outs)

    def info(self) -> dict:
        v, a = C.c_int64(), C.c_int64()
        lm, cp, ep = C.c_int(), C.c_int(), C.c_int()
        ms = C.c_double()
        _check(_lib.sg_batch_info(self.handle, C.byref(v), C.byref(a), C.byref(lm), C.byref(cp), C.byref(ep),
                                  C.byref(ms)))
        return {"vertices": v.value, "arcs": a.value, "light_max": lm.value, "compact_per_sm": cp.value,
                "enum_per_sm": ep.value, "tuned_ms": ms.value}

    def _release(self):
        for g in self._outs:
            g.free()
        self._outs = []

    def free(self):
        if getattr(self, "handle", None):
            self._release()
            _lib.sg_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
