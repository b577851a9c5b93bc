"""ORACLE -- test infrastructure only.

Plain FP64 CPU implementation of Static, DF and DF-P PageRank (arXiv
2404.08299: Eq. 1, Eq. 2, Alg. static, Alg. frontier, Alg. update,
Alg. partition, Alg. affected), of the graph construction and batch update it
relies on, and of the weighted multi-column personalised PageRank and its
adjoint. The arithmetic lives in `oracle.c`; this module only marshals numpy
arrays.

Only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
may import this package. It shares no code with the GPU library.

Parity status: every function here is pinned by `tests/test_oracle_*.py`
(dense direct solves, closed forms, invariants, brute-force set definitions,
finite differences); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ALPHA = 0.85       # damping factor (Section 5.1.2)
TOL = 1e-10        # iteration tolerance, L-inf (Section 5.1.2)
TAU_F = 1e-6       # frontier tolerance (Section 5.1.2)
TAU_P = 1e-6       # prune tolerance (Section 5.1.2)
MAX_ITER = 500     # MAX_ITERATIONS (Section 5.1.2)


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, OpenMP if available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.check_call(base[:2] + ["-fopenmp"] + base[2:], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, _LIB)
    return _LIB


class _Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("final_delta", ctypes.c_double)]


@dataclass
class Stats:
    iterations: int
    converged: bool
    final_delta: float


def _l():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64, ci = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.oracle_csr_build.restype = i64
        lib.oracle_csr_build.argtypes = [i32, i64, P, P, ci, P, P]
        lib.oracle_apply_batch.restype = i64
        lib.oracle_apply_batch.argtypes = [i32, P, P, P, P, i64, P, P, i64, P, P, P, P]
        lib.oracle_partition.argtypes = [i32, P, ci, P, P, P]
        lib.oracle_initial_affected.argtypes = [i32, P, P, P, i64, P, P, i64, P, P]
        lib.oracle_expand_affected.argtypes = [i32, P, P, P, P]
        lib.oracle_pagerank_static.argtypes = [i32, P, P, P, f64, f64, ci, P, P, P]
        lib.oracle_pagerank_dfp.argtypes = [i32, P, P, P, P, P, P, P, i64, P, P, i64, P, f64, f64, f64, f64, ci,
                                            ci, P, P, P, P]
        lib.oracle_pagerank_dt.argtypes = [i32, P, P, P, P, P, P, P, i64, P, P, i64, P, f64, f64, ci, P, P, P, P, P]
        lib.oracle_row_normalise.argtypes = [i32, P, P, P]
        lib.oracle_ppr.argtypes = [i32, ci, P, P, P, P, f64, f64, ci, P, P, P]
        lib.oracle_ppr_adjoint.argtypes = [i32, ci, P, P, P, P, P, P, f64, f64, ci, P, P, P, P]
        lib.oracle_num_threads.restype = ci
        lib.oracle_set_threads.argtypes = [ci]
        _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype)


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(k: int) -> None:
    """OpenMP thread count of later oracle calls."""
    _l().oracle_set_threads(int(k))


def num_threads() -> int:
    return int(_l().oracle_num_threads())


# ---------------------------------------------------------------- graphs ----

def csr_build(n: int, rows, cols, self_loops: bool = True):
    """CSR (off int64[n+1], adj int32[m]) of unique{(rows[i], cols[i])} u {(v, v)}."""
    rows = _c(rows, np.int32)
    cols = _c(cols, np.int32)
    off = np.empty(n + 1, np.int64)
    adj = np.empty(len(rows) + (n if self_loops else 0) + 1, np.int32)
    m = _l().oracle_csr_build(n, len(rows), _p(rows), _p(cols), int(self_loops), _p(off), _p(adj))
    if m < 0:
        raise ValueError("vertex id out of range")
    return off, adj[:m].copy()


@dataclass
class Graph:
    n: int
    out_off: np.ndarray
    out_adj: np.ndarray
    in_off: np.ndarray
    in_adj: np.ndarray

    @property
    def m(self) -> int:
        return int(self.out_off[-1])

    @property
    def outdeg(self) -> np.ndarray:
        return np.diff(self.out_off)

    @property
    def indeg(self) -> np.ndarray:
        return np.diff(self.in_off)


def graph(n: int, src, dst) -> Graph:
    """G (out-CSR) and its transpose G' (in-CSR), deduplicated, with self-loops."""
    oo, oa = csr_build(n, src, dst)
    io, ia = csr_build(n, dst, src)
    return Graph(n, oo, oa, io, ia)


def csr_to_edges(off, adj):
    """(rows, cols) of a CSR, in slot order."""
    n = len(off) - 1
    rows = np.repeat(np.arange(n, dtype=np.int32), np.diff(off))
    return rows, np.asarray(adj, np.int32)


def apply_batch(g: Graph, del_src, del_dst, ins_src, ins_dst):
    """New Graph for E^t = (E^{t-1} \\ D) u I, plus the effectiveness masks of D and I."""
    n = g.n
    ds, dd = _c(del_src, np.int32), _c(del_dst, np.int32)
    is_, id_ = _c(ins_src, np.int32), _c(ins_dst, np.int32)
    noff = np.empty(n + 1, np.int64)
    nadj = np.empty(g.m + len(is_) + 1, np.int32)
    de = np.zeros(max(len(ds), 1), np.uint8)
    ie = np.zeros(max(len(is_), 1), np.uint8)
    m = _l().oracle_apply_batch(n, _p(g.out_off), _p(g.out_adj), _p(ds), _p(dd), len(ds), _p(is_), _p(id_),
                                len(is_), _p(noff), _p(nadj), _p(de), _p(ie))
    if m < 0:
        raise ValueError("vertex id out of range")
    nadj = nadj[:m].copy()
    rows, cols = csr_to_edges(noff, nadj)
    io, ia = csr_build(n, cols, rows)
    return Graph(n, noff, nadj, io, ia), de[:len(ds)].copy(), ie[:len(is_)].copy()


def partition(off, thresholds):
    """Stable degree partition (Alg. partition generalised to len(thresholds)+1 classes)."""
    off = _c(off, np.int64)
    n = len(off) - 1
    thr = _c(thresholds, np.int64)
    P = np.empty(max(n, 1), np.int32)
    cnt = np.empty(len(thr) + 1, np.int64)
    _l().oracle_partition(n, _p(off), len(thr), _p(thr), _p(P), _p(cnt))
    return P[:n].copy(), cnt


# -------------------------------------------------------------- frontier ----

def initial_affected(n, del_src, del_dst, ins_src, del_mask=None, ins_mask=None):
    ds, dd, is_ = _c(del_src, np.int32), _c(del_dst, np.int32), _c(ins_src, np.int32)
    dm = None if del_mask is None else _c(del_mask, np.uint8)
    im = None if ins_mask is None else _c(ins_mask, np.uint8)
    dV = np.zeros(n, np.uint8)
    dN = np.zeros(n, np.uint8)
    _l().oracle_initial_affected(n, _p(ds), _p(dd), _p(dm), len(ds), _p(is_), _p(im), len(is_), _p(dV), _p(dN))
    return dV, dN


def expand_affected(out_off, out_adj, dN, dV):
    """Returns a new deltaV: dV OR out-neighbours of every u with dN[u]."""
    out_off = _c(out_off, np.int64)
    n = len(out_off) - 1
    dVn = np.array(dV, np.uint8, copy=True)
    _l().oracle_expand_affected(n, _p(out_off), _p(_c(out_adj, np.int32)), _p(_c(dN, np.uint8)), _p(dVn))
    return dVn


# ----------------------------------------------------------------- ranks ----

def pagerank_static(g: Graph, alpha=ALPHA, tol=TOL, max_iter=MAX_ITER, R0=None):
    """Alg. static (R0=None) or Alg. naive (R0 = previous ranks). Returns (R, Stats)."""
    R = np.empty(g.n, np.float64)
    st = _Stats()
    r0 = None if R0 is None else _c(R0, np.float64)
    outdeg = _c(g.outdeg, np.int64)
    _l().oracle_pagerank_static(g.n, _p(g.in_off), _p(g.in_adj), _p(outdeg), alpha, tol, max_iter, _p(r0),
                                _p(R), ctypes.byref(st))
    return R, Stats(st.iterations, bool(st.converged), st.final_delta)


def static_ref(g: Graph, alpha=ALPHA):
    """The paper's reference Static run: tau = 1e-100, at most 500 iterations (Section 5.1.4)."""
    return pagerank_static(g, alpha, 1e-100, 500)


def pagerank_dfp(g: Graph, del_src, del_dst, ins_src, Rprev, del_mask=None, ins_mask=None, alpha=ALPHA, tol=TOL,
                 tau_f=TAU_F, tau_p=TAU_P, max_iter=MAX_ITER, prune=True):
    """Alg. frontier with Alg. update / Alg. affected (DF-P if prune else DF).

    Returns (R, Stats, final deltaV, affected count before each sweep).
    """
    n = g.n
    ds, dd, is_ = _c(del_src, np.int32), _c(del_dst, np.int32), _c(ins_src, np.int32)
    dm = None if del_mask is None else _c(del_mask, np.uint8)
    im = None if ins_mask is None else _c(ins_mask, np.uint8)
    R = np.empty(n, np.float64)
    dV = np.empty(n, np.uint8)
    trace = np.zeros(max_iter, np.int64)
    st = _Stats()
    _l().oracle_pagerank_dfp(n, _p(g.out_off), _p(g.out_adj), _p(g.in_off), _p(g.in_adj), _p(ds), _p(dd), _p(dm),
                             len(ds), _p(is_), _p(im), len(is_), _p(_c(Rprev, np.float64)), alpha, tol, tau_f, tau_p,
                             max_iter, int(prune), _p(R), _p(dV), _p(trace), ctypes.byref(st))
    return R, Stats(st.iterations, bool(st.converged), st.final_delta), dV, trace[:st.iterations].copy()


def pagerank_dt(g: Graph, del_src, del_dst, ins_src, Rprev, del_mask=None, ins_mask=None, alpha=ALPHA, tol=TOL,
                max_iter=MAX_ITER):
    """Alg. traversal (Dynamic Traversal): reachability closure of the affected set, then Eq. 1 on it.

    Returns (R, Stats, deltaV after the closure, |deltaV|, closure rounds).
    """
    n = g.n
    ds, dd, is_ = _c(del_src, np.int32), _c(del_dst, np.int32), _c(ins_src, np.int32)
    dm = None if del_mask is None else _c(del_mask, np.uint8)
    im = None if ins_mask is None else _c(ins_mask, np.uint8)
    R = np.empty(n, np.float64)
    dV = np.empty(n, np.uint8)
    na = ctypes.c_int64()
    nr = ctypes.c_int64()
    st = _Stats()
    _l().oracle_pagerank_dt(n, _p(g.out_off), _p(g.out_adj), _p(g.in_off), _p(g.in_adj), _p(ds), _p(dd), _p(dm),
                            len(ds), _p(is_), _p(im), len(is_), _p(_c(Rprev, np.float64)), alpha, tol, max_iter,
                            _p(R), _p(dV), ctypes.byref(na), ctypes.byref(nr), ctypes.byref(st))
    return R, Stats(st.iterations, bool(st.converged), st.final_delta), dV, na.value, nr.value


# ------------------------------------------------- weighted PPR + adjoint ----

def row_normalise(g: Graph, w_out):
    """P_uv = w_uv / sum_k w_uk, in out-CSR slot order."""
    w = _c(w_out, np.float64)
    P = np.empty_like(w)
    _l().oracle_row_normalise(g.n, _p(g.out_off), _p(w), _p(P))
    return P


def out_to_in_perm(g: Graph):
    """perm such that in-CSR slot j holds out-CSR slot perm[j] (same edge)."""
    rows, cols = csr_to_edges(g.out_off, g.out_adj)
    # in-CSR order: by (col, row) ascending
    order = np.lexsort((rows, cols))
    return order


def ppr(g: Graph, P_out, S, alpha=ALPHA, tol=TOL, max_iter=MAX_ITER, R0=None):
    """K-column personalised PageRank with transition weights P (out-CSR order). Returns (R [n,K], Stats)."""
    S = _c(S, np.float64)
    n, K = S.shape
    Pin = _c(np.asarray(P_out, np.float64)[out_to_in_perm(g)], np.float64)
    R = np.empty((n, K), np.float64)
    st = _Stats()
    r0 = None if R0 is None else _c(R0, np.float64)
    _l().oracle_ppr(n, K, _p(g.in_off), _p(g.in_adj), _p(Pin), _p(S), alpha, tol, max_iter, _p(r0), _p(R),
                    ctypes.byref(st))
    return R, Stats(st.iterations, bool(st.converged), st.final_delta)


def ppr_adjoint(g: Graph, w_out, P_out, R, Gw, alpha=ALPHA, tol=TOL, max_iter=MAX_ITER):
    """(lambda, dL/dS, dL/dw in out-CSR order, Stats) for L = sum_c Gw[:, c] . R[:, c]."""
    R = _c(R, np.float64)
    Gw = _c(Gw, np.float64)
    n, K = R.shape
    lam = np.empty((n, K), np.float64)
    gS = np.empty((n, K), np.float64)
    gw = np.empty(g.m, np.float64)
    st = _Stats()
    _l().oracle_ppr_adjoint(n, K, _p(g.out_off), _p(g.out_adj), _p(_c(w_out, np.float64)), _p(_c(P_out, np.float64)),
                            _p(R), _p(Gw), alpha, tol, max_iter, _p(lam), _p(gS), _p(gw), ctypes.byref(st))
    return lam, gS, gw, Stats(st.iterations, bool(st.converged), st.final_delta)
