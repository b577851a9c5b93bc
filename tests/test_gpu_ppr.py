"""K-column weighted personalised PageRank against the FP64 oracle: mixed
precision (FP32 sweeps + FP64 iterative refinement) and plain FP64 both meet
L-inf <= 1e-8; every column tile width gives the same answer; with unit
weights and a uniform teleport column the problem is Static PageRank."""
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


def weighted_case(scale, nsamp, seed, hub=False):
    n, s, d = synth.rmat(scale, nsamp, seed=seed)
    if hub:  # large in-rows: vertex 0 gets up to 6000 sources, vertex 1 up to 5120
        k0, k1 = min(n - 1, 6000), min(n - 2, 5120)
        s = np.concatenate([s, np.arange(1, k0 + 1, dtype=np.int32), np.arange(2, k1 + 2, dtype=np.int32)])
        d = np.concatenate([d, np.zeros(k0, np.int32), np.ones(k1, np.int32)])
    loops = np.arange(n, dtype=np.int32)
    s2, d2 = np.concatenate([s, loops]), np.concatenate([d, loops])
    w = synth.edge_weights(s2, d2, seed=seed)
    g = prdf().Graph(n, dev(s2), dev(d2), dev(w))
    og = oracle.graph(n, s2, d2)
    rows, cols = oracle.csr_to_edges(og.out_off, og.out_adj)
    w_out = synth.edge_weights(rows, cols, seed=seed).astype(np.float64)
    return n, g, og, w_out


@pytest.mark.parametrize("precision", [1, 0])
# (11, .., hub): rows of about 2000 in-edges (warp-per-vertex class); (13, .., hub):
# rows above 4096 in-edges, cut into several 1024-edge chunks
@pytest.mark.parametrize("scale,nsamp,K,hub", [(8, 3000, 5, False), (10, 12000, 64, False), (11, 20000, 17, True),
                                               (13, 60000, 12, True)])
def test_ppr_matches_oracle(precision, scale, nsamp, K, hub):
    n, g, og, w_out = weighted_case(scale, nsamp, seed=scale, hub=hub)
    S = synth.ppr_seeds(n, K, n_seed=16 if n > 100 else 4, seed=3)
    R, st = g.pagerank_ppr(dev(S), precision=precision)
    P = oracle.row_normalise(og, w_out)
    Ro, _ = oracle.ppr(og, P, S, tol=1e-15, max_iter=1000)
    err = np.max(np.abs(host(R) - Ro))
    assert err <= 1e-8, err
    assert st.converged
    if precision == 1:
        assert st.iterations_fp32 > 0 and st.iterations - st.iterations_fp32 <= 4
    assert np.max(np.abs(host(R).sum(axis=0) - 1.0)) <= 1e-8


@pytest.mark.parametrize("tile", [8, 16, 32, 64])
def test_ppr_tile_widths_agree(tile):
    n, g, og, w_out = weighted_case(10, 12000, seed=4, hub=True)
    S = synth.ppr_seeds(n, 40, n_seed=16, seed=5)
    R0, _ = g.pagerank_ppr(dev(S), precision=0, tile=8)
    R, _ = g.pagerank_ppr(dev(S), precision=0, tile=tile)
    assert float((R - R0).abs().max()) <= 1e-12


def test_ppr_unit_weights_uniform_teleport_is_static():
    n, s, d = synth.rmat(10, 12000, seed=6)
    g = prdf().Graph(n, dev(s), dev(d), dev(np.ones(len(s), np.float32)))
    S = np.full((n, 1), 1.0 / n)
    R, st = g.pagerank_ppr(dev(S), precision=1, tol=1e-12)
    ref, _ = oracle.static_ref(oracle.graph(n, s, d))
    assert np.max(np.abs(host(R)[:, 0] - ref)) <= 1e-11


def test_ppr_needs_weights_and_columns():
    n, s, d = synth.rmat(6, 300, seed=1)
    g = prdf().Graph(n, dev(s), dev(d))
    with pytest.raises(prdf().PrdfError) as e:
        g.pagerank_ppr(torch.zeros((n, 2), dtype=torch.float64, device="cuda"))
    assert e.value.code == -5
    gw = prdf().Graph(n, dev(s), dev(d), dev(np.ones(len(s), np.float32)))
    with pytest.raises(prdf().PrdfError):
        gw.pagerank_ppr(torch.zeros((n, 2), dtype=torch.float64, device="cuda"), tile=12)


def test_autotune_tile_is_valid_and_consistent():
    n, g, og, w_out = weighted_case(10, 12000, seed=8, hub=False)
    S = dev(synth.ppr_seeds(n, 24, n_seed=16, seed=9))
    tile = g.autotune_tile(S, sweeps=2)
    assert tile in (8, 16, 32, 64)
    R0, _ = g.pagerank_ppr(S, precision=0, tile=8)
    R1, _ = g.pagerank_ppr(S, precision=0, tile=tile)
    assert float((R1 - R0).abs().max()) <= 1e-12


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("extra_row", [0, 1])
def test_ppr_compact_and_dense_teleport(precision, extra_row):
    """A teleport with non-zero entries on at most n/4 vertices is read through a compact row table (a 4-byte
    index per vertex instead of its whole row); one vertex more keeps the dense form. Both sides of the
    switch meet L-inf 1e-8 against the oracle, and every column still sums to 1."""
    n, g, og, w_out = weighted_case(11, 20000, seed=11)
    K = 8
    rows = np.arange(0, n, 4)[: n // 4]
    if extra_row:
        rows = np.concatenate([rows, [1]])
    S = np.zeros((n, K))
    S[rows, :] = synth.uniform((len(rows), K), seed=21) + 0.01
    S[:, 3] = 0.0
    S[rows[:5], 3] = 1.0  # a column on five seeds only
    S /= S.sum(axis=0, keepdims=True)
    R, st = g.pagerank_ppr(dev(S), precision=precision)
    P = oracle.row_normalise(og, w_out)
    Ro, _ = oracle.ppr(og, P, S, tol=1e-15, max_iter=1000)
    assert np.max(np.abs(host(R) - Ro)) <= 1e-8
    assert st.converged
    assert np.max(np.abs(host(R).sum(axis=0) - 1.0)) <= 1e-8


@pytest.mark.parametrize("precision", [1, 0])
def test_ppr_graph_and_host_loops_give_the_same_bits(precision):
    """The K-column loops run as CUDA graphs (default) or from the host (time_sweeps=1): forward ranks and
    both gradients are bit-identical, with the same sweep counts."""
    n, g, og, w_out = weighted_case(11, 20000, seed=5, hub=True)
    S = dev(synth.ppr_seeds(n, 12, n_seed=16, seed=4))
    G = dev(synth.normal((n, 12), seed=6))
    Rg, stg = g.pagerank_ppr(S, precision=precision)
    Rh, sth = g.pagerank_ppr(S, precision=precision, time_sweeps=1)
    assert torch.equal(Rg, Rh) and stg.iterations == sth.iterations and stg.iterations_fp32 == sth.iterations_fp32
    gSg, gwg, _ = g.pagerank_backward(Rg, G, precision=precision)
    gSh, gwh, _ = g.pagerank_backward(Rg, G, precision=precision, time_sweeps=1)
    assert torch.equal(gSg, gSh) and torch.equal(gwg, gwh)
