"""Python binding of libprdf: Static and DF-P PageRank on one GB300.

Argument marshalling only: every step runs in the hand-written CUDA kernels
of libprdf.so (see include/prdf.h for the C ABI). Tensors are torch CUDA
tensors; work is issued on torch's current CUDA stream. If the library has
not been built, importing works but every call raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libprdf.so")

PRDF_OUT, PRDF_IN = 0, 1
PRDF_FP64, PRDF_FP32_REFINE = 0, 1
PRDF_ACC_EXACT, PRDF_ACC_FP64 = 0, 1
PRDF_ADD_SELF_LOOPS = 1

NOALLOC_MAX_N = 1 << 24  # vertex limit of the fixed scratch of prdf_partition_noalloc

_ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ESTATE"}


class PrdfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("prdf error %d (%s): %s" % (code, _ERRORS.get(code, "?"), msg))
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("tol", ctypes.c_double), ("tau_f", ctypes.c_double),
                ("tau_p", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("tol_fp32_rel", ctypes.c_double), ("accumulate", ctypes.c_int), ("prune", ctypes.c_int),
                ("check_every", ctypes.c_int), ("time_sweeps", ctypes.c_int), ("tile", ctypes.c_int),
                ("expand_pull", ctypes.c_double), ("expand_list", ctypes.c_int64), ("stream", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("final_delta", ctypes.c_double),
                ("iterations_fp32", ctypes.c_int), ("sweeps_launched", ctypes.c_int), ("ms_total", ctypes.c_float),
                ("ms_partition", ctypes.c_float), ("ms_mark", ctypes.c_float), ("ms_iterate", ctypes.c_float),
                ("ms_sweep", ctypes.c_float), ("edges_processed", ctypes.c_longlong),
                ("affected_initial", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong)]


@dataclass
class Stats:
    iterations: int
    converged: bool
    final_delta: float
    iterations_fp32: int
    sweeps_launched: int
    ms_total: float
    ms_partition: float
    ms_mark: float
    ms_iterate: float
    ms_sweep: float
    edges_processed: int
    affected_initial: int
    kernel_launches: int


_lib = None

# exported symbol -> (restype, argtypes)
_P = ctypes.c_void_p
_I32, _I64, _INT, _U = ctypes.c_int32, ctypes.c_int64, ctypes.c_int, ctypes.c_uint
_SIGNATURES = {
    "prdf_params_default": (None, [_P]),
    "prdf_last_error": (ctypes.c_char_p, []),
    "prdf_strerror": (ctypes.c_char_p, [_INT]),
    "prdf_release_cached_memory": (_INT, []),
    "prdf_graph_create": (_INT, [_I32, _P, _P, _P, _I64, _U, _P, _P]),
    "prdf_graph_destroy": (None, [_P]),
    "prdf_graph_size": (_INT, [_P, _P, _P]),
    "prdf_graph_export_csr": (_INT, [_P, _INT, _P, _P, _P, _P]),
    "prdf_graph_apply_batch": (_INT, [_P, _P, _P, _I64, _P, _P, _P, _I64, _P, _P, _P]),
    "prdf_graph_set_thresholds": (_INT, [_P, _INT, _INT, _P]),
    "prdf_partition": (_INT, [_P, _INT, _P, _P, _P]),
    "prdf_partition_noalloc": (_INT, [_P, _I32, _INT, _P, _P, _P, _P]),
    "prdf_initial_affected": (_INT, [_P, _P, _P, _P, _I64, _P, _P, _I64, _P, _P, _P]),
    "prdf_expand_affected": (_INT, [_P, _P, _P, _P]),
    "prdf_pagerank_static": (_INT, [_P, _P, _P, _P, _P]),
    "prdf_pagerank_dfp": (_INT, [_P, _P, _P, _P, _I64, _P, _P, _I64, _P, _P, _P, _P, _P]),
    "prdf_pagerank_dt": (_INT, [_P, _P, _P, _P, _I64, _P, _P, _I64, _P, _P, _P, _P, _P]),
    "prdf_pagerank_ppr": (_INT, [_P, _P, _INT, _P, _P, _P]),
    "prdf_graph_set_weights": (_INT, [_P, _P, _P]),
    "prdf_autotune": (_INT, [_P, _P, _INT, _P, _P]),
    "prdf_autotune_tile": (_INT, [_P, _P, _INT, _P, _INT, _P]),
    "prdf_pagerank_backward": (_INT, [_P, _P, _P, _INT, _P, _P, _P, _P]),
}


def lib():
    """Load libprdf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libprdf.so is not built (run paper_2404_08299_gb300.build.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int):
    if code != 0:
        raise PrdfError(code, lib().prdf_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=None, numel=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, got %d" % (name, numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _stats(s: _Stats) -> Stats:
    return Stats(s.iterations, bool(s.converged), s.final_delta, s.iterations_fp32, s.sweeps_launched, s.ms_total,
                 s.ms_partition, s.ms_mark, s.ms_iterate, s.ms_sweep, s.edges_processed, s.affected_initial,
                 s.kernel_launches)


def params(**kw) -> _Params:
    p = _Params()
    lib().prdf_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    p.stream = _stream()
    return p


def release_cached_memory():
    """Return the device memory the library keeps reserved in its pool for later calls
    (prdf_release_cached_memory); synchronises the current device first."""
    torch.cuda.synchronize()
    _check(lib().prdf_release_cached_memory())


def partition_noalloc(off: torch.Tensor, thresholds):
    """Alg. partition of a device CSR offset array without any device allocation
    (prdf_partition_noalloc). Returns (P int32[n], class sizes)."""
    n = off.numel() - 1
    if not 1 <= n <= NOALLOC_MAX_N:
        raise ValueError("partition_noalloc needs 1 <= n <= %d, got n = %d" % (NOALLOC_MAX_N, n))
    if not 1 <= len(thresholds) <= 3:
        raise ValueError("partition_noalloc takes 1 to 3 thresholds")
    P = torch.empty(n, dtype=torch.int32, device="cuda")
    thr = (ctypes.c_int64 * len(thresholds))(*[int(t) for t in thresholds])
    counts = (ctypes.c_int64 * 4)()
    _check(lib().prdf_partition_noalloc(_ptr(off, torch.int64, name="off"), n, len(thresholds), thr, _ptr(P), counts,
                                        _stream()))
    return P, list(counts)[:len(thresholds) + 1]


class Graph:
    """Device CSR of G and G' (prdf_graph_create)."""

    def __init__(self, n: int, src: torch.Tensor, dst: torch.Tensor, w: torch.Tensor | None = None,
                 self_loops: bool = True):
        m0 = src.numel()
        h = ctypes.c_void_p()
        _check(lib().prdf_graph_create(n, _ptr(src, torch.int32, name="src"), _ptr(dst, torch.int32, m0, "dst"),
                                       _ptr(w, torch.float32, m0, "w"), m0,
                                       PRDF_ADD_SELF_LOOPS if self_loops else 0, _stream(), ctypes.byref(h)))
        self._h = h
        self.weighted = w is not None and m0 > 0  # an empty tensor passes NULL: an unweighted graph

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.prdf_graph_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def size(self):
        n = ctypes.c_int32()
        m = ctypes.c_int64()
        _check(lib().prdf_graph_size(self._h, ctypes.byref(n), ctypes.byref(m)))
        return n.value, m.value

    @property
    def n(self) -> int:
        return self.size()[0]

    @property
    def m(self) -> int:
        return self.size()[1]

    def export_csr(self, which: int = PRDF_OUT):
        n, m = self.size()
        off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        adj = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
        w = torch.empty(max(m, 1), dtype=torch.float32, device="cuda") if self.weighted else None
        _check(lib().prdf_graph_export_csr(self._h, which, _ptr(off), _ptr(adj), _ptr(w), _stream()))
        return off, adj[:m], (w[:m] if w is not None else None)

    def apply_batch(self, del_src, del_dst, ins_src, ins_dst, ins_w=None):
        """Set-semantics batch update; returns (del_eff, ins_eff) uint8 masks."""
        nd, ni = del_src.numel(), ins_src.numel()
        de = torch.zeros(max(nd, 1), dtype=torch.uint8, device="cuda")
        ie = torch.zeros(max(ni, 1), dtype=torch.uint8, device="cuda")
        _check(lib().prdf_graph_apply_batch(self._h, _ptr(del_src, torch.int32, name="del_src"),
                                            _ptr(del_dst, torch.int32, nd, "del_dst"), nd,
                                            _ptr(ins_src, torch.int32, name="ins_src"),
                                            _ptr(ins_dst, torch.int32, ni, "ins_dst"),
                                            _ptr(ins_w, torch.float32, ni, "ins_w"), ni, _ptr(de), _ptr(ie),
                                            _stream()))
        return de[:nd], ie[:ni]

    def autotune(self, sweeps: int = 8, **kw):
        """Pick the fastest in-degree class thresholds for this graph (prdf_autotune).
        Returns (candidate index, ms per sweep)."""
        idx = ctypes.c_int()
        ms = ctypes.c_float()
        p = params(**kw)
        _check(lib().prdf_autotune(self._h, ctypes.byref(p), sweeps, ctypes.byref(idx), ctypes.byref(ms)))
        return idx.value, ms.value

    def autotune_tile(self, S: torch.Tensor, sweeps: int = 3, **kw) -> int:
        """Fastest column tile width for K-column calls with teleport S (prdf_autotune_tile)."""
        tile = ctypes.c_int()
        p = params(**kw)
        _check(lib().prdf_autotune_tile(self._h, _ptr(S, torch.float64, name="S"), S.shape[1], ctypes.byref(p), sweeps,
                                        ctypes.byref(tile)))
        return tile.value

    def set_thresholds(self, which: int, thresholds):
        arr = (ctypes.c_int64 * len(thresholds))(*[int(t) for t in thresholds])
        _check(lib().prdf_graph_set_thresholds(self._h, which, len(thresholds), arr))

    def partition(self, which: int = PRDF_IN):
        n = self.n
        P = torch.empty(n, dtype=torch.int32, device="cuda")
        counts = (ctypes.c_int64 * 8)()
        _check(lib().prdf_partition(self._h, which, _ptr(P), counts, _stream()))
        return P, list(counts)

    def initial_affected(self, del_src, del_dst, ins_src, dV, dN, del_mask=None, ins_mask=None):
        nd, ni = del_src.numel(), ins_src.numel()
        _check(lib().prdf_initial_affected(self._h, _ptr(del_src, torch.int32), _ptr(del_dst, torch.int32, nd),
                                           _ptr(del_mask, torch.uint8, nd), nd, _ptr(ins_src, torch.int32),
                                           _ptr(ins_mask, torch.uint8, ni), ni, _ptr(dV, torch.uint8),
                                           _ptr(dN, torch.uint8), _stream()))

    def expand_affected(self, dN, dV):
        _check(lib().prdf_expand_affected(self._h, _ptr(dN, torch.uint8), _ptr(dV, torch.uint8), _stream()))

    def pagerank_static(self, R0=None, **kw):
        """Alg. static (R0 None) or Naive-dynamic (R0 = previous ranks). Returns (ranks float64[n], Stats)."""
        n = self.n
        R = torch.empty(n, dtype=torch.float64, device="cuda")
        st = _Stats()
        p = params(**kw)
        _check(lib().prdf_pagerank_static(self._h, ctypes.byref(p), _ptr(R0, torch.float64, n, "R0"), _ptr(R),
                                          ctypes.byref(st)))
        return R, _stats(st)

    def pagerank_dfp(self, del_src, del_dst, ins_src, prev_ranks, del_mask=None, ins_mask=None, want_dV=False, **kw):
        """Alg. frontier (DF-P; prune=0 gives DF). Returns (ranks, Stats, final deltaV or None)."""
        n = self.n
        nd, ni = del_src.numel(), ins_src.numel()
        R = torch.empty(n, dtype=torch.float64, device="cuda")
        dV = torch.empty(n, dtype=torch.uint8, device="cuda") if want_dV else None
        st = _Stats()
        p = params(**kw)
        _check(lib().prdf_pagerank_dfp(self._h, _ptr(del_src, torch.int32), _ptr(del_dst, torch.int32, nd),
                                       _ptr(del_mask, torch.uint8, nd), nd, _ptr(ins_src, torch.int32),
                                       _ptr(ins_mask, torch.uint8, ni), ni,
                                       _ptr(prev_ranks, torch.float64, n, "prev_ranks"), _ptr(R), ctypes.byref(p),
                                       _ptr(dV), ctypes.byref(st)))
        return R, _stats(st), dV

    def pagerank_dt(self, del_src, del_dst, ins_src, prev_ranks, del_mask=None, ins_mask=None, want_dV=False, **kw):
        """Alg. traversal (Dynamic Traversal). Returns (ranks, Stats, closed deltaV or None)."""
        n = self.n
        nd, ni = del_src.numel(), ins_src.numel()
        R = torch.empty(n, dtype=torch.float64, device="cuda")
        dV = torch.empty(n, dtype=torch.uint8, device="cuda") if want_dV else None
        st = _Stats()
        p = params(**kw)
        _check(lib().prdf_pagerank_dt(self._h, _ptr(del_src, torch.int32), _ptr(del_dst, torch.int32, nd),
                                      _ptr(del_mask, torch.uint8, nd), nd, _ptr(ins_src, torch.int32),
                                      _ptr(ins_mask, torch.uint8, ni), ni,
                                      _ptr(prev_ranks, torch.float64, n, "prev_ranks"), _ptr(R), ctypes.byref(p),
                                      _ptr(dV), ctypes.byref(st)))
        return R, _stats(st), dV

    def pagerank_ppr(self, S: torch.Tensor, **kw):
        """K-column weighted personalised PageRank (prdf_pagerank_ppr). S: float64 [n, K] on the GPU.
        Returns (R float64 [n, K], Stats)."""
        n = self.n
        if S.dim() != 2 or S.shape[0] != n:
            raise ValueError("S must have shape [n, K]")
        K = S.shape[1]
        R = torch.empty((n, K), dtype=torch.float64, device="cuda")
        st = _Stats()
        p = params(**kw)
        _check(lib().prdf_pagerank_ppr(self._h, _ptr(S, torch.float64, name="S"), K, _ptr(R), ctypes.byref(p),
                                       ctypes.byref(st)))
        return R, _stats(st)

    def set_weights(self, w: torch.Tensor):
        """Edge weights in the out-CSR slot order (float32 [m])."""
        _check(lib().prdf_graph_set_weights(self._h, _ptr(w, torch.float32, self.m, "w"), _stream()))
        self.weighted = True

    def pagerank_backward(self, R: torch.Tensor, G: torch.Tensor, want_grad_S: bool = True, want_grad_w: bool = True,
                          **kw):
        """Adjoint of pagerank_ppr for L = sum(G * R): returns (grad_S [n, K] or None, grad_w [m] or None, Stats)."""
        n, m = self.size()
        K = G.shape[1]
        gS = torch.empty((n, K), dtype=torch.float64, device="cuda") if want_grad_S else None
        gw = torch.empty(max(m, 1), dtype=torch.float64, device="cuda") if want_grad_w else None
        st = _Stats()
        p = params(**kw)
        _check(lib().prdf_pagerank_backward(self._h, _ptr(R, torch.float64, n * K, "R"), _ptr(G, torch.float64, n * K, "G"),
                                            K, _ptr(gS), _ptr(gw), ctypes.byref(p), ctypes.byref(st)))
        return gS, (gw[:m] if gw is not None else None), _stats(st)


class PageRankFn(torch.autograd.Function):
    """R = PageRankFn.apply(graph, S, w, params): K-column weighted personalised PageRank
    (forward: prdf_pagerank_ppr) with gradients for S and the edge weights w (out-CSR slot
    order, float32) from the hand-written adjoint (prdf_pagerank_backward)."""

    @staticmethod
    def forward(ctx, graph, S, w, kw=None):
        kw = dict(kw or {})
        graph.set_weights(w.detach().to(torch.float32).contiguous())
        R, _ = graph.pagerank_ppr(S.detach().to(torch.float64).contiguous(), **kw)
        ctx.graph = graph
        ctx.kw = kw
        ctx.w_dtype = w.dtype
        ctx.S_dtype = S.dtype
        ctx.save_for_backward(R)
        return R

    @staticmethod
    def backward(ctx, grad_R):
        (R,) = ctx.saved_tensors
        need_S, need_w = ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        gS, gw, _ = ctx.graph.pagerank_backward(R, grad_R.detach().to(torch.float64).contiguous(), want_grad_S=need_S,
                                                want_grad_w=need_w, **ctx.kw)
        return (None, gS.to(ctx.S_dtype) if gS is not None else None, gw.to(ctx.w_dtype) if gw is not None else None,
                None)


# Module-level entry points, one per method of the paper (each is the Graph method of the same job).

def static(graph: Graph, R0=None, **kw):
    """Alg. static (R0 None) or Naive-dynamic (Alg. naive, R0 = previous ranks): (ranks, Stats)."""
    return graph.pagerank_static(R0, **kw)


def dfp(graph: Graph, del_src, del_dst, ins_src, prev_ranks, **kw):
    """Alg. frontier, DF-P (prune=0 gives DF), on a graph already holding G^t: (ranks, Stats, deltaV or None)."""
    return graph.pagerank_dfp(del_src, del_dst, ins_src, prev_ranks, **kw)


def dt(graph: Graph, del_src, del_dst, ins_src, prev_ranks, **kw):
    """Alg. traversal (Dynamic Traversal) on a graph already holding G^t: (ranks, Stats, deltaV or None)."""
    return graph.pagerank_dt(del_src, del_dst, ins_src, prev_ranks, **kw)


def ppr(graph: Graph, S, **kw):
    """K-column weighted personalised PageRank: (R [n, K], Stats)."""
    return graph.pagerank_ppr(S, **kw)
