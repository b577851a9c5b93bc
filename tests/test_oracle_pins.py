"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests compares the oracle with itself: each checks it against a
dense direct solve, a closed form, an invariant of the iteration, a
brute-force set definition, finite differences, or the constants the paper
prints (tests/golden/paper_constants.txt).
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------- helpers ----

def dense_P(g):
    """Row-stochastic transition matrix P[u, v] = 1/|out(u)| for (u, v) in E."""
    P = np.zeros((g.n, g.n))
    for u in range(g.n):
        nb = g.out_adj[g.out_off[u]:g.out_off[u + 1]]
        P[u, nb] = 1.0 / len(nb)
    return P


def dense_pagerank(g, alpha=0.85):
    """Direct solve of (I - alpha P^T) r = (1 - alpha)/n (Eq. 1 at its fixed point)."""
    P = dense_P(g)
    A = np.eye(g.n) - alpha * P.T
    return np.linalg.solve(A, np.full(g.n, (1 - alpha) / g.n))


def small_graphs():
    out = []
    rng = np.random.default_rng(7)
    for n in (4, 7, 16, 33, 64):
        m = 3 * n
        src = rng.integers(0, n, m)
        dst = rng.integers(0, n, m)
        out.append(("random%d" % n, n, src, dst))
    n, s, d = synth.rmat(5, 200, seed=3)
    out.append(("rmat5", n, s, d))
    n = 40
    out.append(("chain", n, np.arange(n - 1), np.arange(1, n)))
    out.append(("hub_in", n, np.arange(1, n), np.zeros(n - 1, int)))
    out.append(("hub_out", n, np.zeros(n - 1, int), np.arange(1, n)))
    out.append(("isolated", 5, np.array([], int), np.array([], int)))
    return out


# ------------------------------------------------------------ constants ----

def test_defaults_are_the_papers_constants():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    assert oracle.ALPHA == vals["alpha"]
    assert oracle.TOL == vals["tau"]
    assert oracle.TAU_F == vals["tau_f"]
    assert oracle.TAU_P == vals["tau_p"]
    assert oracle.MAX_ITER == vals["max_iterations"]


# ------------------------------------------------------------- graphs -----

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_csr_build_matches_set_definition(seed):
    n = 50
    src = synth.randint(400, n, seed)
    dst = synth.randint(400, n, seed + 100)
    off, adj = oracle.csr_build(n, src, dst)
    E = set(zip(src.tolist(), dst.tolist())) | {(v, v) for v in range(n)}
    for u in range(n):
        row = adj[off[u]:off[u + 1]].tolist()
        assert row == sorted({v for (a, v) in E if a == u})
    assert off[-1] == len(E)


def test_csr_build_rejects_bad_ids():
    with pytest.raises(ValueError):
        oracle.csr_build(4, np.array([0, 4]), np.array([1, 1]))
    with pytest.raises(ValueError):
        oracle.csr_build(4, np.array([0, -1]), np.array([1, 1]))


def test_transpose_is_transpose():
    n, s, d = synth.rmat(7, 900, seed=5)
    g = oracle.graph(n, s, d)
    out_e = set(zip(*[x.tolist() for x in oracle.csr_to_edges(g.out_off, g.out_adj)]))
    in_e = {(b, a) for (a, b) in zip(*[x.tolist() for x in oracle.csr_to_edges(g.in_off, g.in_adj)])}
    assert out_e == in_e


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_apply_batch_set_semantics(seed):
    n = 40
    g = oracle.graph(n, synth.randint(300, n, seed), synth.randint(300, n, seed + 9))
    E0 = set(zip(*[x.tolist() for x in oracle.csr_to_edges(g.out_off, g.out_adj)]))
    ds, dd, is_, id_ = synth.batch(n, g.out_off, g.out_adj, 60, seed=seed)
    # add adversarial entries: a self-loop deletion, a deleted-and-reinserted pair, a duplicate insertion,
    # an insertion of an existing edge, a deletion of a missing edge
    e_any = next(iter(sorted(E0 - {(v, v) for v in range(n)})))
    missing = next((u, v) for u in range(n) for v in range(n) if (u, v) not in E0)
    ds = np.concatenate([ds, [3, e_any[0], missing[0]]]).astype(np.int32)
    dd = np.concatenate([dd, [3, e_any[1], missing[1]]]).astype(np.int32)
    is_ = np.concatenate([is_, [e_any[0], is_[0], e_any[0]]]).astype(np.int32)
    id_ = np.concatenate([id_, [e_any[1], id_[0], e_any[1]]]).astype(np.int32)
    g1, dm, im = oracle.apply_batch(g, ds, dd, is_, id_)
    D = {(a, b) for a, b in zip(ds.tolist(), dd.tolist()) if a != b}
    I = set(zip(is_.tolist(), id_.tolist()))
    E1 = ((E0 - D) | I) | {(v, v) for v in range(n)}
    got = set(zip(*[x.tolist() for x in oracle.csr_to_edges(g1.out_off, g1.out_adj)]))
    assert got == E1
    for i, (a, b) in enumerate(zip(ds.tolist(), dd.tolist())):
        assert dm[i] == int((a, b) in E0 and (a, b) not in E1)
    for i, (a, b) in enumerate(zip(is_.tolist(), id_.tolist())):
        assert im[i] == int((a, b) not in E0 and (a, b) in E1)
    # the deleted-and-reinserted existing edge is in neither effective list
    assert e_any in E1
    # transpose of the new graph
    in_e = {(b, a) for (a, b) in zip(*[x.tolist() for x in oracle.csr_to_edges(g1.in_off, g1.in_adj)])}
    assert in_e == E1


@pytest.mark.parametrize("thr", [[2], [0], [100], [1, 3], [2, 4, 8]])
def test_partition_brute_force(thr):
    n, s, d = synth.rmat(6, 300, seed=11)
    g = oracle.graph(n, s, d)
    deg = g.indeg
    P, cnt = oracle.partition(g.in_off, thr)

    def cls(v):
        return sum(deg[v] > t for t in thr)

    assert P.tolist() == sorted(range(n), key=lambda v: (cls(v), v))
    assert cnt.tolist() == [sum(cls(v) == c for v in range(n)) for c in range(len(thr) + 1)]


def test_initial_and_expand_affected_sets():
    n = 30
    g = oracle.graph(n, synth.randint(120, n, 21), synth.randint(120, n, 22))
    ds, dd = np.array([1, 5, 7], np.int32), np.array([2, 6, 9], np.int32)
    is_ = np.array([11, 12], np.int32)
    dmask = np.array([1, 0, 1], np.uint8)
    dV, dN = oracle.initial_affected(n, ds, dd, is_, del_mask=dmask)
    assert set(np.flatnonzero(dN)) == {1, 7, 11, 12}
    assert set(np.flatnonzero(dV)) == {2, 9}
    dV2 = oracle.expand_affected(g.out_off, g.out_adj, dN, dV)
    want = {2, 9}
    for u in (1, 7, 11, 12):
        want |= set(g.out_adj[g.out_off[u]:g.out_off[u + 1]].tolist())
    assert set(np.flatnonzero(dV2)) == want
    assert {1, 7, 11, 12} <= want  # self-loops: a marked source marks itself


# -------------------------------------------------------------- static ----

@pytest.mark.parametrize("name,n,src,dst", small_graphs())
def test_static_ref_matches_dense_solve(name, n, src, dst):
    g = oracle.graph(n, src, dst)
    R, st = oracle.static_ref(g)
    r = dense_pagerank(g)
    assert np.max(np.abs(R - r)) <= 1e-12, name


@pytest.mark.parametrize("name,n,src,dst", small_graphs())
def test_static_tol_stops_at_first_small_delta(name, n, src, dst):
    g = oracle.graph(n, src, dst)
    R, st = oracle.pagerank_static(g)
    assert st.converged and st.final_delta <= 1e-10
    # the iterate one step earlier had not converged (iterations are reproducible from 1/n)
    if st.iterations > 1:
        _, st2 = oracle.pagerank_static(g, max_iter=st.iterations - 1)
        assert st2.final_delta > 1e-10
    # error of the tol-stopped result is within the geometric tail bound alpha/(1-alpha) * tau (L-inf)
    assert np.max(np.abs(R - dense_pagerank(g))) <= 0.85 / 0.15 * 1e-10 * n


@pytest.mark.parametrize("n", [1, 2, 5, 64, 1000])
def test_directed_cycle_is_uniform(n):
    src = np.arange(n)
    dst = (src + 1) % n
    g = oracle.graph(n, src, dst)
    R, st = oracle.static_ref(g)
    assert np.max(np.abs(R * n - 1.0)) <= 1e-13


@pytest.mark.parametrize("k", [1, 3, 10, 50])
def test_bidirectional_star_closed_form(k):
    n = k + 1
    src = np.concatenate([np.zeros(k, int), np.arange(1, n)])
    dst = np.concatenate([np.arange(1, n), np.zeros(k, int)])
    g = oracle.graph(n, src, dst)
    R, _ = oracle.static_ref(g)
    a, b = 0.85, 0.15 / n
    # leaf: r_l (1 - a/2) = a r_c/(k+1) + b ; centre: r_c (1 - a/(k+1)) = k a r_l / 2 + b
    rc = (1 - k * b / (1 - a / 2)) / (1 + k * a / ((k + 1) * (1 - a / 2)))
    rl = (a * rc / (k + 1) + b) / (1 - a / 2)
    assert abs(R[0] - rc) <= 1e-14
    assert np.max(np.abs(R[1:] - rl)) <= 1e-14
    assert abs(rc + k * rl - 1) <= 1e-14


@pytest.mark.parametrize("k", [1, 4, 20])
def test_out_star_closed_form(k):
    n = k + 1
    g = oracle.graph(n, np.zeros(k, int), np.arange(1, n))
    R, _ = oracle.static_ref(g)
    a, b = 0.85, 0.15 / n
    rc = b / (1 - a / (k + 1))
    rl = (a * rc / (k + 1) + b) / (1 - a)
    assert abs(R[0] - rc) <= 1e-14
    assert np.max(np.abs(R[1:] - rl)) <= 1e-14


@pytest.mark.parametrize("iters", [1, 2, 7, 30])
def test_rank_mass_is_one_every_iterate(iters):
    n, s, d = synth.rmat(10, 8000, seed=4)
    g = oracle.graph(n, s, d)
    R, st = oracle.pagerank_static(g, tol=0.0, max_iter=iters)
    assert st.iterations == iters
    assert abs(R.sum() - 1.0) <= n * 1e-15


def test_l1_contraction():
    n, s, d = synth.rmat(9, 5000, seed=8)
    g = oracle.graph(n, s, d)
    its = [oracle.pagerank_static(g, tol=0.0, max_iter=k)[0] for k in range(1, 12)]
    its.insert(0, np.full(n, 1.0 / n))
    diffs = [np.abs(its[k + 1] - its[k]).sum() for k in range(len(its) - 1)]
    for k in range(1, len(diffs)):
        assert diffs[k] <= 0.85 * diffs[k - 1] + 1e-15


def test_naive_dynamic_from_fixed_point_stops_at_once():
    n, s, d = synth.rmat(8, 2000, seed=2)
    g = oracle.graph(n, s, d)
    R, _ = oracle.static_ref(g)
    R2, st = oracle.pagerank_static(g, R0=R)
    assert st.iterations == 1 and np.max(np.abs(R2 - R)) <= 1e-15


# ---------------------------------------------------------------- DF-P ----

def _batch_graphs(seed, scale=8, nsamp=3000, size=40):
    n, s, d = synth.rmat(scale, nsamp, seed=seed)
    g0 = oracle.graph(n, s, d)
    ds, dd, is_, id_ = synth.batch(n, g0.out_off, g0.out_adj, size, seed=seed, s1=1)
    g1, dm, im = oracle.apply_batch(g0, ds, dd, is_, id_)
    return g0, g1, (ds, dd, is_, id_, dm, im)


def test_dfp_fixed_point_identity():
    """Eq. 2 rearranges to Eq. 1 when every vertex has one self-loop: r* is a fixed point of the DF-P update."""
    g0, g1, _ = _batch_graphs(1)
    r = dense_pagerank(g1)
    n = g1.n
    allv = np.arange(n, dtype=np.int32)
    # inserting (u, .) for every u marks every vertex affected through the self-loops
    R, st, dV, trace = oracle.pagerank_dfp(g1, [], [], allv, r, tau_p=0.0)
    assert trace[0] == n
    assert st.iterations == 1
    assert np.max(np.abs(R - r)) <= 1e-16 * 50


def test_dfp_empty_batch_is_identity():
    g0, g1, _ = _batch_graphs(2)
    R1, _ = oracle.pagerank_static(g1)
    R, st, dV, trace = oracle.pagerank_dfp(g1, [], [], [], R1)
    assert trace[0] == 0 and st.iterations == 1
    assert np.array_equal(R, R1)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dfp_close_to_static_ref_after_batch(seed):
    """A vertex is pruned once its relative change is <= tau_p; with contraction factor alpha the remaining
    relative error of a pruned vertex is about alpha/(1-alpha) * tau_p, which bounds every vertex's relative
    error and hence the L1 error (ranks sum to 1). With tight tolerances DF-P reaches the reference Static
    ranks."""
    g0, g1, (ds, dd, is_, id_, dm, im) = _batch_graphs(seed, scale=10, nsamp=12000, size=30)
    R0, _ = oracle.pagerank_static(g0)
    R, st, dV, trace = oracle.pagerank_dfp(g1, ds, dd, is_, R0, del_mask=dm, ins_mask=im)
    ref, _ = oracle.static_ref(g1)
    bound = 0.85 / 0.15 * 1e-6
    assert np.max(np.abs(R - ref) / ref) <= bound
    assert np.abs(R - ref).sum() <= bound
    assert trace[0] < g1.n  # the frontier starts small
    assert abs(R.sum() - 1) <= 1e-5
    Rt, st, _, _ = oracle.pagerank_dfp(g1, ds, dd, is_, R0, del_mask=dm, ins_mask=im, tau_f=1e-13, tau_p=1e-13,
                                       tol=1e-14)
    assert np.abs(Rt - ref).sum() <= 1e-10


def test_dfp_small_batch_on_larger_graph_within_prune_bound():
    """2^14-vertex R-MAT with a 10-edge batch: the frontier spreads through most of the graph (small diameter),
    so the L1 error is governed by the same alpha/(1-alpha) * tau_p bound; it stays far below the error of
    the stale ranks R^{t-1}."""
    g0, g1, (ds, dd, is_, id_, dm, im) = _batch_graphs(7, scale=14, nsamp=1 << 18, size=10)
    R0, _ = oracle.pagerank_static(g0)
    R, st, dV, trace = oracle.pagerank_dfp(g1, ds, dd, is_, R0, del_mask=dm, ins_mask=im)
    ref, _ = oracle.static_ref(g1)
    err = np.abs(R - ref).sum()
    assert err <= 0.85 / 0.15 * 1e-6
    assert err <= 0.05 * np.abs(R0 - ref).sum()


def test_df_all_affected_equals_naive_dynamic():
    """With every vertex affected and tau_f = 0 (always expand), DF runs Eq. 1 on all vertices: Alg. naive."""
    g0, g1, _ = _batch_graphs(3)
    R0, _ = oracle.pagerank_static(g0)
    allv = np.arange(g1.n, dtype=np.int32)
    R, st, _, trace = oracle.pagerank_dfp(g1, [], [], allv, R0, tau_f=-1.0, prune=False)
    Rn, stn = oracle.pagerank_static(g1, R0=R0)
    assert np.all(trace == g1.n)
    assert st.iterations == stn.iterations
    assert np.array_equal(R, Rn)


def test_dfp_full_frontier_converges_to_dense_solution():
    g0, g1, _ = _batch_graphs(4)
    R0, _ = oracle.pagerank_static(g0)
    allv = np.arange(g1.n, dtype=np.int32)
    R, st, _, _ = oracle.pagerank_dfp(g1, [], [], allv, R0, tau_f=-1.0, tau_p=-1.0, tol=1e-15)
    assert np.max(np.abs(R - dense_pagerank(g1))) <= 1e-13


def test_dfp_prune_everything_leaves_no_affected():
    """tau_p = 1 prunes every processed vertex (relative change is at most 1); the final sweep is not followed
    by an expansion, so deltaV ends empty."""
    g0, g1, (ds, dd, is_, id_, dm, im) = _batch_graphs(5)
    R0, _ = oracle.pagerank_static(g0)
    R, st, dV, trace = oracle.pagerank_dfp(g1, ds, dd, is_, R0, del_mask=dm, ins_mask=im, tau_p=1.0)
    assert dV.sum() == 0


def test_dfp_unaffected_vertices_keep_their_rank():
    g0, g1, (ds, dd, is_, id_, dm, im) = _batch_graphs(6)
    R0, _ = oracle.pagerank_static(g0)
    R, st, dV, trace = oracle.pagerank_dfp(g1, ds, dd, is_, R0, del_mask=dm, ins_mask=im, max_iter=1)
    dV0, dN0 = oracle.initial_affected(g1.n, ds, dd, is_, dm, im)
    aff = oracle.expand_affected(g1.out_off, g1.out_adj, dN0, dV0).astype(bool)
    assert np.array_equal(R[~aff], R0[~aff])
    assert trace[0] == aff.sum()


# ------------------------------------------------------ Dynamic Traversal ----

def _reachable(g, seeds):
    """Brute-force breadth-first search along out-edges from a set of seed vertices."""
    seen = np.zeros(g.n, bool)
    stack = [int(v) for v in seeds]
    for v in stack:
        seen[v] = True
    while stack:
        u = stack.pop()
        for w in g.out_adj[g.out_off[u]:g.out_off[u + 1]]:
            if not seen[w]:
                seen[w] = True
                stack.append(int(w))
    return seen


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dt_affected_set_is_the_reachable_set(seed):
    """Alg. traversal marks every vertex reachable in G^t from the batch: the targets of effective deletions and
    the out-neighbours of the sources of effective deletions and insertions, then everything they reach."""
    g0, g1, (ds, dd, is_, id_, dm, im) = _batch_graphs(seed, scale=7, nsamp=300, size=6)
    R0, _ = oracle.pagerank_static(g0)
    R, st, dV, na, rounds = oracle.pagerank_dt(g1, ds, dd, is_, R0, del_mask=dm, ins_mask=im)
    dm, im = dm.astype(bool), im.astype(bool)
    seeds = set(np.asarray(dd)[dm].tolist())
    for u in list(np.asarray(ds)[dm]) + list(np.asarray(is_)[im]):
        seeds.update(g1.out_adj[g1.out_off[u]:g1.out_off[u + 1]].tolist())
    reach = _reachable(g1, sorted(seeds))
    assert np.array_equal(dV.astype(bool), reach)
    assert na == reach.sum()
    assert 0 < reach.sum() < g1.n  # a sparse random graph: the closure is a proper subset


def test_dt_reaches_the_exact_ranks_and_keeps_the_rest():
    """Vertices not reachable from the batch keep their exact rank (PageRank of v depends only on the vertices
    that reach v), so from the exact ranks of G^{t-1} DT converges to the exact ranks of G^t, and every
    unaffected vertex is left bit-for-bit unchanged."""
    g0, g1, (ds, dd, is_, id_, dm, im) = _batch_graphs(4, scale=7, nsamp=300, size=6)
    r0 = dense_pagerank(g0)
    R, st, dV, na, rounds = oracle.pagerank_dt(g1, ds, dd, is_, r0, del_mask=dm, ins_mask=im, tol=1e-15)
    aff = dV.astype(bool)
    assert np.array_equal(R[~aff], r0[~aff])
    assert np.max(np.abs(R - dense_pagerank(g1))) <= 1e-13


def test_dt_on_a_strongly_connected_graph_is_naive_dynamic():
    """When every vertex reaches every other, the closure is all of V and DT runs Eq. 1 on every vertex, which
    is Alg. naive."""
    n, s, d = synth.rmat(7, 500, seed=5)
    ring = np.arange(n)
    s = np.concatenate([s, ring])
    d = np.concatenate([d, (ring + 1) % n])
    g0 = oracle.graph(n, s, d)
    ds, dd, is_, id_ = synth.batch(n, g0.out_off, g0.out_adj, 8, seed=5, s1=1)
    g1, dm, im = oracle.apply_batch(g0, ds, dd, is_, id_)
    # keep the ring: the batch's deletions must not break strong connectivity
    keep = ~((np.asarray(dd) == (np.asarray(ds) + 1) % n))
    ds, dd, dm = np.asarray(ds)[keep], np.asarray(dd)[keep], np.asarray(dm)[keep]
    g1, dm2, im = oracle.apply_batch(g0, ds, dd, is_, id_)
    R0, _ = oracle.pagerank_static(g0)
    R, st, dV, na, rounds = oracle.pagerank_dt(g1, ds, dd, is_, R0, del_mask=dm2, ins_mask=im)
    Rn, stn = oracle.pagerank_static(g1, R0=R0)
    assert na == n
    assert st.iterations == stn.iterations
    assert np.array_equal(R, Rn)


def test_dt_empty_batch_is_identity():
    g0, g1, _ = _batch_graphs(2)
    R1, _ = oracle.pagerank_static(g1)
    R, st, dV, na, rounds = oracle.pagerank_dt(g1, [], [], [], R1)
    assert na == 0 and dV.sum() == 0
    assert st.iterations == 1 and st.final_delta == 0
    assert np.array_equal(R, R1)


# ------------------------------------------------------- PPR + adjoint ----

def _weighted(seed=1, scale=6, nsamp=500):
    n, s, d = synth.rmat(scale, nsamp, seed=seed)
    g = oracle.graph(n, s, d)
    rows, cols = oracle.csr_to_edges(g.out_off, g.out_adj)
    w = synth.edge_weights(rows, cols, seed=seed).astype(np.float64)
    return g, w


def dense_Pw(g, w):
    P = np.zeros((g.n, g.n))
    rows, cols = oracle.csr_to_edges(g.out_off, g.out_adj)
    P[rows, cols] = w
    return P / P.sum(axis=1, keepdims=True)


def test_ppr_dense_solve_and_mass():
    g, w = _weighted()
    P = oracle.row_normalise(g, w)
    S = synth.ppr_seeds(g.n, 5, n_seed=4, seed=3)
    R, st = oracle.ppr(g, P, S, tol=1e-15)
    Pd = dense_Pw(g, w)
    Rd = np.linalg.solve(np.eye(g.n) - 0.85 * Pd.T, 0.15 * S)
    assert np.max(np.abs(R - Rd)) <= 1e-13
    assert np.max(np.abs(R.sum(axis=0) - 1)) <= 1e-13


def test_ppr_unweighted_uniform_teleport_is_static_pagerank():
    n, s, d = synth.rmat(7, 1000, seed=9)
    g = oracle.graph(n, s, d)
    P = oracle.row_normalise(g, np.ones(g.m))
    S = np.full((n, 1), 1.0 / n)
    R, _ = oracle.ppr(g, P, S, tol=1e-16, max_iter=500)
    Rs, _ = oracle.static_ref(g)
    assert np.max(np.abs(R[:, 0] - Rs)) <= 1e-15


def test_adjoint_dense_and_identity():
    g, w = _weighted(seed=2)
    P = oracle.row_normalise(g, w)
    K = 3
    S = synth.ppr_seeds(g.n, K, n_seed=4, seed=5)
    R, _ = oracle.ppr(g, P, S, tol=1e-15)
    Gw = synth.normal((g.n, K), seed=6)
    lam, gS, gw, st = oracle.ppr_adjoint(g, w, P, R, Gw, tol=1e-15)
    Pd = dense_Pw(g, w)
    lam_d = np.linalg.solve(np.eye(g.n) - 0.85 * Pd, Gw)
    assert np.max(np.abs(lam - lam_d)) <= 1e-12
    assert np.max(np.abs(gS - 0.15 * lam_d)) <= 1e-12
    # sum_k P_uk lambda[k] = (lambda[u] - g[u]) / alpha
    assert np.max(np.abs(Pd @ lam - (lam - Gw) / 0.85)) <= 1e-12


def test_adjoint_matches_central_differences():
    g, w = _weighted(seed=3, scale=5, nsamp=200)
    K = 2
    S = synth.ppr_seeds(g.n, K, n_seed=3, seed=7)
    Gw = synth.normal((g.n, K), seed=8)

    def loss(S_, w_):
        R_, _ = oracle.ppr(g, oracle.row_normalise(g, w_), S_, tol=1e-15, max_iter=2000)
        return float((Gw * R_).sum())

    P = oracle.row_normalise(g, w)
    R, _ = oracle.ppr(g, P, S, tol=1e-15, max_iter=2000)
    lam, gS, gw, _ = oracle.ppr_adjoint(g, w, P, R, Gw, tol=1e-15, max_iter=2000)
    h = 1e-6
    rng = np.random.default_rng(0)
    for (v, c) in [(int(rng.integers(g.n)), int(rng.integers(K))) for _ in range(6)]:
        Sp, Sm = S.copy(), S.copy()
        Sp[v, c] += h
        Sm[v, c] -= h
        fd = (loss(Sp, w) - loss(Sm, w)) / (2 * h)
        assert abs(fd - gS[v, c]) <= 1e-5 * max(1e-3, abs(fd)), (v, c, fd, gS[v, c])
    for j in rng.choice(g.m, 8, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[j] += h
        wm[j] -= h
        fd = (loss(S, wp) - loss(S, wm)) / (2 * h)
        assert abs(fd - gw[j]) <= 1e-5 * max(1e-4, abs(fd)), (j, fd, gw[j])
