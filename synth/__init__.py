"""Seeded synthetic inputs (graphs, batch updates, personalisation, loss weights).

Shared by the oracle tests, the GPU tests and the benchmark. This module draws
inputs only; it contains none of the PageRank arithmetic. The C source
(`synth.c`) documents the counter-based SplitMix64 streams used.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

RMAT_ABC = (0.57, 0.19, 0.19)  # (a, b, c); d = 0.05


def build(force: bool = False) -> str:
    """Compile libsynth.so next to its source (gcc, OpenMP if available)."""
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


def _l():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.synth_key.restype = u64
        lib.synth_key.argtypes = [u64, u64, u64, u64]
        lib.synth_draw.restype = u64
        lib.synth_draw.argtypes = [u64, u64]
        lib.synth_rmat.argtypes = [ctypes.c_int, i64, f64, f64, f64, u64, P, P]
        lib.synth_grid.restype = i64
        lib.synth_grid.argtypes = [ctypes.c_int, f64, u64, P, P]
        lib.synth_batch.restype = i64
        lib.synth_batch.argtypes = [i32, P, P, i64, i64, u64, u64, u64, P, P, P, P]
        lib.synth_edge_weights.argtypes = [i64, P, P, u64, f64, f64, P]
        lib.synth_ppr_seeds.argtypes = [i32, ctypes.c_int, ctypes.c_int, u64, P]
        lib.synth_normal.argtypes = [i64, u64, P]
        lib.synth_uniform.argtypes = [i64, u64, P]
        lib.synth_randint.argtypes = [i64, i64, u64, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def rmat(scale: int, nedges: int, seed: int = 1, abc=RMAT_ABC):
    """Raw R-MAT samples (duplicates and u == v pairs included): (n, src, dst)."""
    src = np.empty(nedges, np.int32)
    dst = np.empty(nedges, np.int32)
    _l().synth_rmat(scale, nedges, abc[0], abc[1], abc[2], seed, _p(src), _p(dst))
    return 1 << scale, src, dst


def grid(side: int, p_drop: float = 0.05, seed: int = 1):
    """side x side bidirectional 4-neighbour grid with dropped edges: (n, src, dst)."""
    cap = 4 * side * side
    src = np.empty(cap, np.int32)
    dst = np.empty(cap, np.int32)
    m = _l().synth_grid(side, p_drop, seed, _p(src), _p(dst))
    return side * side, src[:m].copy(), dst[:m].copy()


def batch(n: int, off: np.ndarray, adj: np.ndarray, size: int, seed: int = 1, s1: int = 0, s2: int = 0,
          ins_frac: float = 0.8):
    """Random batch of `size` updates (round(ins_frac*size) insertions, rest deletions).

    Returns (del_src, del_dst, ins_src, ins_dst) as int32 arrays.
    """
    off = np.ascontiguousarray(off, np.int64)
    adj = np.ascontiguousarray(adj, np.int32)
    n_ins = int(round(ins_frac * size))
    n_del = size - n_ins
    ds = np.empty(max(n_del, 1), np.int32)
    dd = np.empty(max(n_del, 1), np.int32)
    is_ = np.empty(max(n_ins, 1), np.int32)
    id_ = np.empty(max(n_ins, 1), np.int32)
    got = _l().synth_batch(n, _p(off), _p(adj), n_del, n_ins, seed, s1, s2, _p(ds), _p(dd), _p(is_), _p(id_))
    return ds[:got].copy(), dd[:got].copy(), is_[:n_ins].copy(), id_[:n_ins].copy()


def edge_weights(src: np.ndarray, dst: np.ndarray, seed: int = 1, lo: float = 0.5, hi: float = 1.5):
    w = np.empty(len(src), np.float32)
    _l().synth_edge_weights(len(src), _p(np.ascontiguousarray(src, np.int32)),
                            _p(np.ascontiguousarray(dst, np.int32)), seed, lo, hi, _p(w))
    return w


def ppr_seeds(n: int, K: int, n_seed: int = 16, seed: int = 1):
    """[n, K] float64 personalisation matrix; each column sums to 1."""
    S = np.empty((n, K), np.float64)
    _l().synth_ppr_seeds(n, K, n_seed, seed, _p(S))
    return S


def normal(shape, seed: int = 1):
    out = np.empty(int(np.prod(shape)), np.float64)
    _l().synth_normal(out.size, seed, _p(out))
    return out.reshape(shape)


def uniform(shape, seed: int = 1):
    out = np.empty(int(np.prod(shape)), np.float64)
    _l().synth_uniform(out.size, seed, _p(out))
    return out.reshape(shape)


def randint(count: int, bound: int, seed: int = 1):
    out = np.empty(count, np.int32)
    _l().synth_randint(count, bound, seed, _p(out))
    return out


def key(seed: int, s1: int = 0, s2: int = 0, s3: int = 0) -> int:
    return int(_l().synth_key(seed, s1, s2, s3))


def draw(k: int, i: int) -> int:
    return int(_l().synth_draw(k, i))
