"""The allocation-free partition entry point (prdf_partition_noalloc) gives the
same partition as prdf_partition.

It serves callers that cannot allocate device memory where they partition
(their memory belongs to a pool that owns all of it, or their path must not
take cudaMalloc's device-wide synchronisation); its scratch is a fixed array
inside the library. Partitions are integer outputs, so the check is
bit-exact. Two calls in a row with different sizes and thresholds show that
the scratch shared between calls (which keeps the previous call's contents)
does not leak into the next result. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from helpers import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_08299_gb300 import build
    build.build()
    torch.cuda.init()


def _graph(scale, nsamp, seed):
    import paper_2404_08299_gb300 as prdf
    n, s, d = synth.rmat(scale, nsamp, seed=seed)
    return prdf.Graph(n, dev(s, torch.int32), dev(d, torch.int32))


def test_noalloc_partition_matches_allocating_partition_twice():
    import paper_2404_08299_gb300 as prdf
    cases = [(14, 200000, 1, [8, 64, 2048]), (12, 30000, 2, [2])]  # second call: smaller n, fewer classes
    for scale, nsamp, seed, thr in cases:
        g = _graph(scale, nsamp, seed)
        g.set_thresholds(prdf.PRDF_IN, thr)
        P_ref, cnt_ref = g.partition(prdf.PRDF_IN)
        off, _, _ = g.export_csr(prdf.PRDF_IN)
        # through the C ABI directly
        n = off.numel() - 1
        P = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        thr_arr = (ctypes.c_int64 * len(thr))(*thr)
        counts = (ctypes.c_int64 * 4)()
        rc = prdf.lib().prdf_partition_noalloc(ctypes.c_void_p(off.data_ptr()), n, len(thr), thr_arr,
                                               ctypes.c_void_p(P.data_ptr()), counts,
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, prdf.lib().prdf_last_error()
        assert torch.equal(P, P_ref)
        assert list(counts)[:len(thr) + 1] == cnt_ref[:len(thr) + 1]
        # and through the binding
        P2, cnt2 = prdf.partition_noalloc(off, thr)
        assert torch.equal(P2, P_ref) and cnt2 == cnt_ref[:len(thr) + 1]


def test_noalloc_partition_at_its_size_limit():
    """n = 2^24 exactly with three thresholds (four classes): the last count tiles, the scan's tail and
    the class totals at the top of the fixed scratch are all used. A graph of 2^24 vertices with 2^22
    R-MAT samples spreads the degrees over all four classes; bit-exact against prdf_partition."""
    import paper_2404_08299_gb300 as prdf
    n_max = prdf.NOALLOC_MAX_N
    n, s, d = synth.rmat(24, 1 << 22, seed=4)
    assert n == n_max
    g = prdf.Graph(n, dev(s, torch.int32), dev(d, torch.int32))
    thr = [1, 2, 8]
    for which in (prdf.PRDF_IN, prdf.PRDF_OUT):
        g.set_thresholds(which, thr)
        P_ref, cnt_ref = g.partition(which)
        off, _, _ = g.export_csr(which)
        assert min(cnt_ref[:4]) > 0
        for _ in range(2):
            P, cnt = prdf.partition_noalloc(off, thr)
            assert torch.equal(P, P_ref) and cnt == cnt_ref[:4]
    del g
    with pytest.raises(ValueError):
        prdf.partition_noalloc(torch.zeros(n_max + 2, dtype=torch.int64, device="cuda"), thr)
    with pytest.raises(ValueError):
        prdf.partition_noalloc(torch.zeros(1, dtype=torch.int64, device="cuda"), thr)


def test_noalloc_partition_rejects_sizes_beyond_its_scratch():
    import paper_2404_08299_gb300 as prdf
    off = torch.zeros(2, dtype=torch.int64, device="cuda")
    P = torch.zeros(1, dtype=torch.int32, device="cuda")
    thr = (ctypes.c_int64 * 1)(4)
    counts = (ctypes.c_int64 * 4)()
    rc = prdf.lib().prdf_partition_noalloc(ctypes.c_void_p(off.data_ptr()), (1 << 24) + 1, 1, thr,
                                           ctypes.c_void_p(P.data_ptr()), counts, None)
    assert rc == -1
    assert b"exceeds the fixed scratch limit" in prdf.lib().prdf_last_error()
