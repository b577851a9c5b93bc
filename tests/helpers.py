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


def dynamic_case(seed, scale, nsamp, size, thresholds=None):
    """R-MAT graph on the GPU and in the oracle, R^{t-1} from the oracle, and one random batch
    (80% insertions, 20% deletions) applied on both sides. Returns
    (gpu graph, oracle G^t, R^{t-1} on the GPU, (ds, dd, is, id, gpu masks, oracle masks))."""
    import paper_2404_08299_gb300 as prdf
    n, s, d = synth.rmat(scale, nsamp, seed=seed)
    return batch_case(n, s, d, seed, size, thresholds)


def batch_case(n, s, d, seed, size, thresholds=None, extra=None):
    """As dynamic_case for a given edge list; extra = (ds, dd, is, id) appended to the random batch."""
    import torch
    import paper_2404_08299_gb300 as prdf
    og0 = oracle.graph(n, s, d)
    g = prdf.Graph(n, dev(s, torch.int32), dev(d, torch.int32))
    if thresholds is not None:
        g.set_thresholds(prdf.PRDF_IN, thresholds)
    R0o, _ = oracle.pagerank_static(og0)  # R^{t-1} from the oracle feeds both sides
    ds, dd, is_, id_ = synth.batch(n, og0.out_off, og0.out_adj, size, seed=seed, s1=7)
    if extra is not None:
        ds, dd, is_, id_ = (np.concatenate([a, b]).astype(np.int32) for a, b in zip((ds, dd, is_, id_), extra))
    de, ie = g.apply_batch(dev(ds), dev(dd), dev(is_), dev(id_))
    og1, dmo, imo = oracle.apply_batch(og0, ds, dd, is_, id_)
    return g, og1, dev(R0o), (ds, dd, is_, id_, de, ie, dmo, imo)


def planted_hub_case(seed, size=40):
    """R-MAT with 2^15 vertices plus two planted in-hubs (vertex 7 with about 19 K distinct sources, vertex 11
    with about 7 K), so that rows of in-degree above 4096 (the block-per-vertex class of the DF / DF-P sweep
    under the default thresholds) exist; the batch deletes 16 existing in-edges of each hub and inserts 16 new
    ones on top of `size` random updates."""
    n, s, d = synth.rmat(15, 1 << 18, seed=seed)
    h7 = synth.randint(30000, n, seed=seed + 100)
    h11 = synth.randint(8000, n, seed=seed + 200)
    s = np.concatenate([s, h7, h11]).astype(np.int32)
    d = np.concatenate([d, np.full(30000, 7, np.int32), np.full(8000, 11, np.int32)]).astype(np.int32)
    og0 = oracle.graph(n, s, d)
    eds, edd, eis, eid = [], [], [], []
    for k, h in enumerate((7, 11)):
        row = og0.in_adj[og0.in_off[h]:og0.in_off[h + 1]]
        row = row[row != h]
        pick = row[synth.randint(16, len(row), seed=seed + 300 + k)]
        cand = synth.randint(200, n, seed=seed + 400 + k)
        new = cand[~np.isin(cand, row) & (cand != h)][:16]
        eds.append(pick)
        edd.append(np.full(len(pick), h, np.int32))
        eis.append(new)
        eid.append(np.full(len(new), h, np.int32))
    extra = tuple(np.concatenate(x).astype(np.int32) for x in (eds, edd, eis, eid))
    return n, s, d, extra
