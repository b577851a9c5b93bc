"""GPU parity of the integer parts of the hot path, bit-exact against the oracle:
CSR / transposed CSR build (Section 3.1, 4.3), set-semantics batch update
(Section 3.3), degree partition (Alg. partition), initialAffected and
expandAffected (Alg. affected)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import adversarial_edges, dev, host, huge_row_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_08299_gb300 import build
    build.build()
    torch.cuda.init()


def prdf():
    import paper_2404_08299_gb300 as p
    return p


def gpu_graph(n, src, dst, w=None):
    return prdf().Graph(n, dev(src, torch.int32), dev(dst, torch.int32), None if w is None else dev(w, torch.float32))


def check_csr(g, og):
    P = prdf()
    off, adj, _ = g.export_csr(P.PRDF_OUT)
    assert np.array_equal(host(off), og.out_off)
    assert np.array_equal(host(adj), og.out_adj)
    off, adj, _ = g.export_csr(P.PRDF_IN)
    assert np.array_equal(host(off), og.in_off)
    assert np.array_equal(host(adj), og.in_adj)


def ones(src, weighted):
    """Unit weights for the weighted form of a build: unweighted lists take the radix-sort build,
    weighted ones the per-row sort; both must give the oracle's CSR."""
    return np.ones(len(src), np.float32) if weighted else None


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("name,n,src,dst", adversarial_edges())
def test_csr_build_adversarial(name, n, src, dst, weighted):
    check_csr(gpu_graph(n, src, dst, ones(src, weighted)), oracle.graph(n, src, dst))


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("scale,nsamp", [(10, 16000), (16, 1 << 20)])
def test_csr_build_rmat(scale, nsamp, weighted):
    n, s, d = synth.rmat(scale, nsamp, seed=1)
    check_csr(gpu_graph(n, s, d, ones(s, weighted)), oracle.graph(n, s, d))


@pytest.mark.parametrize("n,m0", [(3, 1), (1000, 4096 - 1000), (1000, 4097 - 1000), (70001, 500000),
                                  ((1 << 17) + 3, 1 << 20), ((1 << 20) + 5, 3000)])
def test_csr_build_radix_sizes(n, m0):
    """Radix-sort build at vertex counts that are not powers of two (key widths of 2 to 18 bits a field,
    one to five passes) and at key counts of exactly one 4096-key tile and one key more; random ids with many
    duplicates and runs of empty rows in the no-self-loop form (the last case is a list far shorter than n,
    whose row offsets are found row-parallel)."""
    rng = np.random.default_rng(n + m0)
    s = (rng.integers(0, n, m0) if n < 1000 else rng.zipf(1.3, m0) % n).astype(np.int32)
    d = rng.integers(0, n, m0).astype(np.int32)
    check_csr(gpu_graph(n, s, d), oracle.graph(n, s, d))
    g = prdf().Graph(n, dev(s), dev(d), self_loops=False)
    P = prdf()
    for which, (r, c) in ((P.PRDF_OUT, (s, d)), (P.PRDF_IN, (d, s))):
        off, adj, _ = g.export_csr(which)
        want_off, want_adj = oracle.csr_build(n, r, c, self_loops=False)
        assert np.array_equal(host(off), want_off) and np.array_equal(host(adj), want_adj)


def test_builds_after_releasing_the_memory_pool():
    """Buffers freed by one graph are reused by the next from the library's pool;
    after the reserve is released a new build still matches the oracle."""
    n, s, d = synth.rmat(12, 60000, seed=4)
    og = oracle.graph(n, s, d)
    for _ in range(2):
        g = gpu_graph(n, s, d)
        check_csr(g, og)
        del g
    prdf().release_cached_memory()
    check_csr(gpu_graph(n, s, d), og)


@pytest.mark.parametrize("weighted", [False, True])
def test_csr_build_grid(weighted):
    n, s, d = synth.grid(128, 0.05, seed=1)
    check_csr(gpu_graph(n, s, d, ones(s, weighted)), oracle.graph(n, s, d))


@pytest.mark.parametrize("weighted", [False, True])
def test_csr_build_bitmap_and_block_rows(weighted):
    n, s, d = huge_row_edges()
    g = gpu_graph(n, s, d, ones(s, weighted))
    og = oracle.graph(n, s, d)
    check_csr(g, og)
    assert np.diff(og.out_off).max() > 16384 and np.diff(og.in_off).max() > 16384


def test_csr_weights_take_max_of_duplicates():
    n, s, d = huge_row_edges(n=1 << 14, hub_deg=30000)
    rng = np.random.default_rng(3)
    w = rng.uniform(0.5, 1.5, len(s)).astype(np.float32)
    g = gpu_graph(n, s, d, w)
    P = prdf()
    for which, (r, c) in ((P.PRDF_OUT, (s, d)), (P.PRDF_IN, (d, s))):
        off, adj, ww = g.export_csr(which)
        off, adj, ww = host(off), host(adj), host(ww)
        best = {}
        for a, b, x in zip(r.tolist(), c.tolist(), w.tolist()):
            best[(a, b)] = max(best.get((a, b), 0.0), x)
        rows = np.repeat(np.arange(n), np.diff(off))
        for a, b, x in zip(rows.tolist(), adj.tolist(), ww.tolist()):
            want = best.get((a, b), 1.0 if a == b else None)
            assert want is not None and np.float32(want) == np.float32(x), (a, b, x, want)


def test_csr_rejects_out_of_range_ids():
    with pytest.raises(prdf().PrdfError) as e:
        gpu_graph(4, np.array([0, 4], np.int32), np.array([1, 1], np.int32))
    assert e.value.code == -1
    with pytest.raises(prdf().PrdfError):
        gpu_graph(4, np.array([0, -1], np.int32), np.array([1, 1], np.int32))


@pytest.mark.parametrize("thr", [[2], [0], [8, 64, 2048], [1, 3], [4, 16]])
def test_partition_bit_exact(thr):
    n, s, d = synth.rmat(12, 60000, seed=2)
    g = gpu_graph(n, s, d)
    og = oracle.graph(n, s, d)
    P = prdf()
    for which, off in ((P.PRDF_IN, og.in_off), (P.PRDF_OUT, og.out_off)):
        g.set_thresholds(which, thr)
        Pg, cnt = g.partition(which)
        Po, cnto = oracle.partition(off, thr)
        assert np.array_equal(host(Pg), Po)
        assert cnt[:len(thr) + 1] == cnto.tolist()


def test_partition_ragged_tiles():
    # n not a multiple of the 2048-vertex tile, one class empty
    n = 2048 * 3 + 77
    s = synth.randint(9000, n, 4)
    d = synth.randint(9000, n, 5)
    g = gpu_graph(n, s, d)
    og = oracle.graph(n, s, d)
    g.set_thresholds(prdf().PRDF_IN, [1000])
    Pg, cnt = g.partition(prdf().PRDF_IN)
    Po, cnto = oracle.partition(og.in_off, [1000])
    assert np.array_equal(host(Pg), Po) and cnt[:2] == cnto.tolist() and cnto[1] == 0


@pytest.mark.parametrize("seed,size,scale,nsamp", [(1, 50, 11, 30000), (2, 400, 11, 30000), (3, 3000, 11, 30000),
                                                   (4, 6000, 15, 1 << 19), (5, 20000, 11, 30000)])
def test_apply_batch_bit_exact(seed, size, scale, nsamp):
    """Batches on both merge forms (in place on the numbering's CSRs while the edges changed since the last
    numbering stay within 1/64 of |E|; on the original-id CSRs with a fresh numbering otherwise) and both batch
    preparations (one block up to 4096 deletions and 4096 insertions; batch CSRs built by the radix sort above:
    sizes 6000 and 20000)."""
    n, s, d = synth.rmat(scale, nsamp, seed=seed)
    g = gpu_graph(n, s, d)
    og = oracle.graph(n, s, d)
    ds, dd, is_, id_ = synth.batch(n, og.out_off, og.out_adj, size, seed=seed, s1=3)
    # adversarial entries: self-loop deletion, deleted+reinserted, duplicate insertion, missing deletion
    e_u = int(np.flatnonzero(np.diff(og.out_off) > 1)[0])
    row = og.out_adj[og.out_off[e_u]:og.out_off[e_u + 1]]
    e_v = int(row[row != e_u][0])
    ds = np.concatenate([ds, [5, e_u, 0]]).astype(np.int32)
    dd = np.concatenate([dd, [5, e_v, n - 1]]).astype(np.int32)
    is_ = np.concatenate([is_, [e_u, is_[0]]]).astype(np.int32)
    id_ = np.concatenate([id_, [e_v, id_[0]]]).astype(np.int32)
    de, ie = g.apply_batch(dev(ds), dev(dd), dev(is_), dev(id_))
    og1, dmo, imo = oracle.apply_batch(og, ds, dd, is_, id_)
    check_csr(g, og1)
    assert np.array_equal(host(de), dmo)
    assert np.array_equal(host(ie), imo)


def test_apply_batch_empty_and_consecutive():
    n, s, d = synth.rmat(10, 12000, seed=9)
    g = gpu_graph(n, s, d)
    og = oracle.graph(n, s, d)
    e = np.zeros(0, np.int32)
    de, ie = g.apply_batch(dev(e), dev(e), dev(e), dev(e))
    check_csr(g, og)
    for b in range(3):
        ds, dd, is_, id_ = synth.batch(n, og.out_off, og.out_adj, 100, seed=9, s1=1, s2=b)
        g.apply_batch(dev(ds), dev(dd), dev(is_), dev(id_))
        og, _, _ = oracle.apply_batch(og, ds, dd, is_, id_)
        check_csr(g, og)


def test_apply_batch_weighted_set_semantics():
    """Weighted rows after a batch: (old \\ D) u I per row; an edge that survives and is inserted again keeps
    the larger weight, a deleted edge inserted again takes the inserted weight, duplicates take their maximum,
    self-loops are never deleted."""
    n, s, d = synth.rmat(10, 8000, seed=21)
    loops = np.arange(n, dtype=np.int32)
    s2, d2 = np.concatenate([s, loops]), np.concatenate([d, loops])
    w0 = synth.edge_weights(s2, d2, seed=21)
    g = gpu_graph(n, s2, d2, w0)
    off, adj, ww = (host(x) for x in g.export_csr(prdf().PRDF_OUT))
    rows = np.repeat(np.arange(n), np.diff(off))
    old = {(int(a), int(b)): float(x) for a, b, x in zip(rows, adj, ww)}
    ds, dd, is_, id_ = synth.batch(n, off, adj, 300, seed=21, s1=2)
    nonself = [(a, b) for (a, b) in old if a != b]
    rng = np.random.default_rng(5)
    keep = [nonself[i] for i in rng.choice(len(nonself), 6, replace=False)]
    ds = np.concatenate([ds, [keep[0][0], keep[1][0], 3]]).astype(np.int32)       # two more deletions + a self-loop
    dd = np.concatenate([dd, [keep[0][1], keep[1][1], 3]]).astype(np.int32)
    is_ = np.concatenate([is_, [keep[0][0], keep[2][0], keep[2][0], 3]]).astype(np.int32)  # re-insert deleted,
    id_ = np.concatenate([id_, [keep[0][1], keep[2][1], keep[2][1], 3]]).astype(np.int32)  # re-insert twice, loop
    iw = rng.uniform(0.5, 1.5, len(is_)).astype(np.float32)
    de, ie = g.apply_batch(dev(ds), dev(dd), dev(is_), dev(id_), ins_w=dev(iw))
    want = dict(old)
    for a, b in zip(ds.tolist(), dd.tolist()):
        if a != b:
            want.pop((a, b), None)
    survivors = set(want)
    ins_best = {}
    for a, b, x in zip(is_.tolist(), id_.tolist(), iw.tolist()):
        ins_best[(a, b)] = max(ins_best.get((a, b), 0.0), x)
    for e, x in ins_best.items():
        want[e] = max(want[e], x) if e in survivors else x
    P = prdf()
    for which, flip in ((P.PRDF_OUT, False), (P.PRDF_IN, True)):
        off1, adj1, w1 = (host(x) for x in g.export_csr(which))
        r1 = np.repeat(np.arange(n), np.diff(off1))
        got = {((int(b), int(a)) if flip else (int(a), int(b))): float(x) for a, b, x in zip(r1, adj1, w1)}
        assert got.keys() == want.keys()
        assert all(np.float32(got[e]) == np.float32(want[e]) for e in want)
        for u in range(n):  # rows stay sorted
            assert np.all(np.diff(adj1[off1[u]:off1[u + 1]]) > 0)
    assert np.array_equal(host(de), np.array([(a, b) in old and a != b and (a, b) not in want for a, b in
                                              zip(ds.tolist(), dd.tolist())], np.uint8))


def test_apply_batch_on_graph_without_self_loops_rebuilds():
    """A graph created without self-loops is rebuilt by a batch update, which gives every vertex its self-loop."""
    n, s, d = synth.rmat(9, 3000, seed=22)
    g = prdf().Graph(n, dev(s), dev(d), self_loops=False)
    og = oracle.graph(n, s, d)
    ds, dd, is_, id_ = synth.batch(n, og.out_off, og.out_adj, 40, seed=22, s1=1)
    g.apply_batch(dev(ds), dev(dd), dev(is_), dev(id_))
    og1, _, _ = oracle.apply_batch(og, ds, dd, is_, id_)
    check_csr(g, og1)


def test_initial_and_expand_affected_bit_exact():
    n, s, d = synth.rmat(13, 120000, seed=4)
    g = gpu_graph(n, s, d)
    og = oracle.graph(n, s, d)
    ds, dd, is_, id_ = synth.batch(n, og.out_off, og.out_adj, 500, seed=4)
    dmask = (np.arange(len(ds)) % 3 != 0).astype(np.uint8)
    dV = torch.zeros(n, dtype=torch.uint8, device="cuda")
    dN = torch.zeros(n, dtype=torch.uint8, device="cuda")
    g.initial_affected(dev(ds), dev(dd), dev(is_), dV, dN, del_mask=dev(dmask))
    dVo, dNo = oracle.initial_affected(n, ds, dd, is_, del_mask=dmask)
    assert np.array_equal(host(dV), dVo) and np.array_equal(host(dN), dNo)
    # expand from identical input flags, for several class splits (thread/warp/block kernels)
    rng = np.random.default_rng(0)
    for thr in ([8, 64, 2048], [2], [0, 1, 4]):
        g.set_thresholds(prdf().PRDF_OUT, thr)
        dN_in = (rng.random(n) < 0.05).astype(np.uint8)
        dV_in = (rng.random(n) < 0.02).astype(np.uint8)
        dVg = dev(dV_in)
        g.expand_affected(dev(dN_in), dVg)
        assert np.array_equal(host(dVg), oracle.expand_affected(og.out_off, og.out_adj, dN_in, dV_in))
