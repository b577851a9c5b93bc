"""Shared helpers of the GPU parity tests: seeded graphs, device transfer, oracle calls."""
import numpy as np
import torch

import oracle
import synth


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def rmat_edges(scale, nsamp, seed=1):
    return synth.rmat(scale, nsamp, seed=seed)


def adversarial_edges():
    """Small edge lists covering the degenerate cases of the method."""
    cases = []
    cases.append(("single_vertex", 1, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    cases.append(("no_edges", 7, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    cases.append(("self_loops_and_dups", 5, np.array([0, 0, 1, 1, 1, 4, 4], np.int32),
                  np.array([0, 1, 2, 2, 2, 4, 0], np.int32)))
    n = 50
    cases.append(("chain", n, np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32)))
    cases.append(("in_hub", 3000, np.arange(1, 3000, dtype=np.int32), np.zeros(2999, np.int32)))
    cases.append(("out_hub", 3000, np.zeros(2999, np.int32), np.arange(1, 3000, dtype=np.int32)))
    return cases


def huge_row_edges(n=1 << 15, hub_deg=40000, seed=5):
    """A vertex with more than 16384 raw entries (bitmap path) plus duplicates, and a
    mid-size row (shared-memory bitonic path)."""
    rng = np.random.default_rng(seed)
    hub_dst = rng.integers(0, n, hub_deg).astype(np.int32)
    mid_dst = rng.integers(0, n, 3000).astype(np.int32)
    rs = rng.integers(0, n, 20000).astype(np.int32)
    rd = rng.integers(0, n, 20000).astype(np.int32)
    src = np.concatenate([np.full(hub_deg, 7, np.int32), np.full(3000, 11, np.int32), rs, hub_dst])
    dst = np.concatenate([hub_dst, mid_dst, rd, np.full(hub_deg, 7, np.int32)])
    return n, src, dst


def csr_equal(off_a, adj_a, off_b, adj_b):
    return np.array_equal(np.asarray(off_a), np.asarray(off_b)) and np.array_equal(np.asarray(adj_a),
                                                                                    np.asarray(adj_b))
