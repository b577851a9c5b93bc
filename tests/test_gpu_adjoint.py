"""Adjoint of the K-column weighted personalised PageRank (hand-written
backward behind torch.autograd): gradients of L = sum_c G_c . R_c with
respect to the teleport matrix S and the edge weights, against the FP64
oracle adjoint, a dense adjoint solve, and central finite differences
(h = 1e-6, FP64) on a 2^10-vertex R-MAT instance with 2^14 samples."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_08299_gb300 import build
    build.build()
    torch.cuda.init()


def prdf():
    import paper_2404_08299_gb300 as p
    return p


def case(scale, nsamp, seed, K, hub=False):
    n, s, d = synth.rmat(scale, nsamp, seed=seed)
    if hub:  # vertex 0 with 6000 in- and out-neighbours: its rows span several 1024-edge chunks
        k = min(n - 1, 6000)
        ks = np.arange(1, k + 1, dtype=np.int32)
        s = np.concatenate([s, ks, np.zeros(k, np.int32)])
        d = np.concatenate([d, np.zeros(k, np.int32), ks])
    loops = np.arange(n, dtype=np.int32)
    s2, d2 = np.concatenate([s, loops]), np.concatenate([d, loops])
    w = synth.edge_weights(s2, d2, seed=seed)
    g = prdf().Graph(n, dev(s2), dev(d2), dev(w))
    og = oracle.graph(n, s2, d2)
    rows, cols = oracle.csr_to_edges(og.out_off, og.out_adj)
    w_out = synth.edge_weights(rows, cols, seed=seed).astype(np.float64)
    S = synth.ppr_seeds(n, K, n_seed=16, seed=seed + 1)
    Gw = synth.normal((n, K), seed=seed + 2)
    return n, g, og, w_out, S, Gw


def dense_P(og, w_out):
    P = np.zeros((og.n, og.n))
    rows, cols = oracle.csr_to_edges(og.out_off, og.out_adj)
    P[rows, cols] = w_out
    return P / P.sum(axis=1, keepdims=True)


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("scale,nsamp,hub", [(10, 1 << 14, False), (13, 60000, True)])
def test_backward_matches_oracle_adjoint(precision, scale, nsamp, hub):
    n, g, og, w_out, S, Gw = case(scale, nsamp, 3, 6, hub=hub)
    # the graph's out-CSR order is the oracle's (both sorted), so weights line up
    off, adj, wg = g.export_csr(prdf().PRDF_OUT)
    assert np.array_equal(host(adj), og.out_adj)
    R, _ = g.pagerank_ppr(dev(S), precision=precision)
    gS, gw, st = g.pagerank_backward(R, dev(Gw), precision=precision)
    P = oracle.row_normalise(og, w_out)
    Ro, _ = oracle.ppr(og, P, S, tol=1e-15, max_iter=2000)
    lam, gSo, gwo, _ = oracle.ppr_adjoint(og, w_out, P, Ro, Gw, tol=1e-15, max_iter=2000)
    assert np.max(np.abs(host(gS) - gSo)) <= 1e-8 * max(1.0, np.abs(gSo).max())
    assert np.max(np.abs(host(gw) - gwo)) <= 1e-8 * max(1.0, np.abs(gwo).max())
    assert st.converged


def test_backward_matches_dense_adjoint():
    n, g, og, w_out, S, Gw = case(8, 3000, 5, 3)
    R, _ = g.pagerank_ppr(dev(S))
    gS, _, _ = g.pagerank_backward(R, dev(Gw), want_grad_w=False)
    Pd = dense_P(og, w_out)
    lam = np.linalg.solve(np.eye(n) - 0.85 * Pd, Gw)
    assert np.max(np.abs(host(gS) - 0.15 * lam)) <= 1e-9


def test_backward_central_differences_2p10():
    """Central differences of the FP64 loss (h = 1e-6): S entries through the GPU FP64 forward,
    weight entries through the FP64 oracle forward (weights are stored in FP32 on the GPU, too
    coarse for a 1e-6 step)."""
    n, g, og, w_out, S, Gw = case(10, 1 << 14, 7, 4)
    R, _ = g.pagerank_ppr(dev(S), precision=0, tol=1e-15, max_iter=3000)
    gS, gw, _ = g.pagerank_backward(R, dev(Gw), precision=0, tol=1e-15, max_iter=3000)
    gS, gw = host(gS), host(gw)
    h = 1e-6
    rng = np.random.default_rng(1)

    def loss_gpu(S_):
        Rx, _ = g.pagerank_ppr(dev(S_), precision=0, tol=1e-15, max_iter=3000)
        return float((host(Rx) * Gw).sum())

    seeds = np.argwhere(S > 0)
    picks = [tuple(seeds[i]) for i in rng.choice(len(seeds), 4, replace=False)]
    picks += [(int(rng.integers(n)), int(rng.integers(S.shape[1]))) for _ in range(2)]
    for (v, c) in picks:
        Sp, Sm = S.copy(), S.copy()
        Sp[v, c] += h
        Sm[v, c] -= h
        fd = (loss_gpu(Sp) - loss_gpu(Sm)) / (2 * h)
        assert abs(fd - gS[v, c]) <= 1e-5 * max(abs(fd), 1e-3), (v, c, fd, gS[v, c])

    def loss_oracle(w_):
        Rx, _ = oracle.ppr(og, oracle.row_normalise(og, w_), S, tol=1e-15, max_iter=3000)
        return float((Rx * Gw).sum())

    for j in rng.choice(og.m, 8, replace=False):
        wp, wm = w_out.copy(), w_out.copy()
        wp[j] += h
        wm[j] -= h
        fd = (loss_oracle(wp) - loss_oracle(wm)) / (2 * h)
        assert abs(fd - gw[j]) <= 1e-5 * max(abs(fd), 1e-4), (j, fd, gw[j])


def test_autograd_function():
    n, g, og, w_out, S, Gw = case(9, 6000, 11, 3)
    _, _, w0 = g.export_csr(prdf().PRDF_OUT)
    St = dev(S).requires_grad_(True)
    wt = w0.clone().requires_grad_(True)
    R = prdf().PageRankFn.apply(g, St, wt, {"precision": 1})
    loss = (R * dev(Gw)).sum()
    loss.backward()
    gS, gw, _ = g.pagerank_backward(R.detach(), dev(Gw), precision=1)  # same options as the autograd call
    assert torch.allclose(St.grad, gS, rtol=0, atol=1e-12)
    assert torch.allclose(wt.grad.double(), gw.float().double(), rtol=1e-6, atol=1e-9)


def test_set_weights_rejects_non_positive():
    n, g, og, w_out, S, Gw = case(6, 300, 1, 2)
    bad = torch.ones(g.m, dtype=torch.float32, device="cuda")
    bad[3] = 0.0
    with pytest.raises(prdf().PrdfError):
        g.set_weights(bad)
