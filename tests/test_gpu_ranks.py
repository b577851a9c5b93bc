"""GPU parity of the floating-point parts of the hot path against the oracle:
Static PageRank (Alg. static, Eq. 1), Naive-dynamic (Alg. naive), DF and DF-P
(Alg. frontier, Alg. update with Eq. 2, Alg. affected).

Tolerances: FP64 static ranks within L-inf 1e-8 of the oracle (the stated
target); both sides run the same Jacobi iteration to the same stop rule, so
in practice they agree to ~1e-15 and the tests also check the iteration count.
DF-P ranks within L1 1e-6 of the oracle's Static ranks where the frontier stays
small, else within the prune bound alpha/(1-alpha)*tau_p (derived in the oracle
pins); step-by-step DF-P parity on small graphs checks flags exactly.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import adversarial_edges, batch_case, dev, dynamic_case, host, planted_hub_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_08299_gb300 import build
    build.build()
    torch.cuda.init()


def prdf():
    import paper_2404_08299_gb300 as p
    return p


def gpu_graph(n, src, dst):
    return prdf().Graph(n, dev(src, torch.int32), dev(dst, torch.int32))


ACC = [0, 1]  # PRDF_ACC_EXACT, PRDF_ACC_FP64


@pytest.mark.parametrize("acc", ACC)
@pytest.mark.parametrize("name,n,src,dst", adversarial_edges())
def test_static_adversarial(acc, name, n, src, dst):
    g = gpu_graph(n, src, dst)
    og = oracle.graph(n, src, dst)
    R, st = g.pagerank_static(accumulate=acc)
    Ro, sto = oracle.pagerank_static(og)
    assert np.max(np.abs(host(R) - Ro)) <= 1e-8
    assert abs(st.iterations - sto.iterations) <= 1 and st.converged


@pytest.mark.parametrize("acc", ACC)
def test_static_rmat_scale16_config(acc):
    """The 2^16-vertex R-MAT configuration: 2^20 samples, seed 1."""
    n, s, d = synth.rmat(16, 1 << 20, seed=1)
    g = gpu_graph(n, s, d)
    og = oracle.graph(n, s, d)
    R, st = g.pagerank_static(accumulate=acc)
    Ro, sto = oracle.pagerank_static(og)
    err = np.max(np.abs(host(R) - Ro))
    assert err <= 1e-8, err
    assert err <= 1e-13  # same iteration, rounding-level differences only
    assert st.iterations == sto.iterations
    assert abs(host(R).sum() - 1.0) <= 1e-12


@pytest.mark.parametrize("thr", [[8, 64, 2048], [1], [0, 4, 16], [100000]])
def test_static_every_class_split_gives_same_bits(thr):
    """Exact accumulation makes every kernel shape produce identical ranks."""
    n, s, d = synth.rmat(12, 80000, seed=3)
    g = gpu_graph(n, s, d)
    R0, _ = g.pagerank_static()
    g.set_thresholds(prdf().PRDF_IN, thr)
    R1, _ = g.pagerank_static()
    assert torch.equal(R0, R1)


def test_static_grid():
    n, s, d = synth.grid(96, 0.05, seed=1)
    g = gpu_graph(n, s, d)
    og = oracle.graph(n, s, d)
    R, st = g.pagerank_static()
    Ro, sto = oracle.pagerank_static(og)
    assert np.max(np.abs(host(R) - Ro)) <= 1e-8
    assert abs(st.iterations - sto.iterations) <= 1


def test_static_max_iter_and_check_cadence():
    n, s, d = synth.rmat(11, 20000, seed=6)
    g = gpu_graph(n, s, d)
    og = oracle.graph(n, s, d)
    for it in (1, 2, 7):
        for ce in (1, 3, 8):
            R, st = g.pagerank_static(max_iter=it, check_every=ce)
            Ro, sto = oracle.pagerank_static(og, max_iter=it)
            assert st.iterations == sto.iterations == it
            assert np.max(np.abs(host(R) - Ro)) <= 1e-14


def test_naive_dynamic_from_previous_ranks():
    n, s, d = synth.rmat(12, 50000, seed=7)
    og = oracle.graph(n, s, d)
    R0 = synth.uniform(n, seed=3)
    R0 /= R0.sum()
    g = gpu_graph(n, s, d)
    R, st = g.pagerank_static(R0=dev(R0))
    Ro, sto = oracle.pagerank_static(og, R0=R0)
    assert np.max(np.abs(host(R) - Ro)) <= 1e-8
    assert abs(st.iterations - sto.iterations) <= 1


def test_static_rejects_bad_params():
    n, s, d = synth.rmat(6, 300, seed=1)
    g = gpu_graph(n, s, d)
    for kw in ({"alpha": 1.0}, {"alpha": 0.0}, {"tol": 0.0}, {"max_iter": 0}, {"alpha": float("nan")},
               {"expand_pull": -1.0}, {"expand_pull": float("nan")}, {"expand_list": -2}):
        with pytest.raises(prdf().PrdfError) as e:
            g.pagerank_static(**kw)
        assert e.value.code == -1


# ------------------------------------------------------------------ DF-P ----

def _dynamic_case(seed, scale, nsamp, size, thresholds=None):
    return dynamic_case(seed, scale, nsamp, size, thresholds)


def _check_dfp_step_by_step(g, og1, R0, batch, prune, expand_pull):
    """expand_list -1 (automatic: off on graphs this small) and 64 (push rounds with at most 64 frontier vertices
    expand from a list, larger ones through the partition kernels): both must give the oracle's trace."""
    ds, dd, is_, id_, de, ie, dmo, imo = batch
    Ro, sto, dVo, trace = oracle.pagerank_dfp(og1, ds, dd, is_, host(R0), del_mask=dmo, ins_mask=imo, prune=bool(prune))
    for expand_list in (-1, 64):
        R, st, dV = g.pagerank_dfp(dev(ds), dev(dd), dev(is_), R0, del_mask=de, ins_mask=ie, want_dV=True,
                                   prune=prune, expand_pull=expand_pull, expand_list=expand_list)
        assert st.iterations == sto.iterations
        assert st.affected_initial == trace[0]
        assert np.array_equal(host(dV), dVo)
        assert np.max(np.abs(host(R) - Ro) / Ro) <= 1e-12


@pytest.mark.parametrize("expand_pull", [1 / 16, 0.0, 2.0])  # automatic, always pull, always push
@pytest.mark.parametrize("prune", [1, 0])
@pytest.mark.parametrize("seed,scale,nsamp,size", [(1, 8, 3000, 20), (2, 10, 12000, 60), (3, 12, 50000, 5)])
def test_dfp_matches_oracle_step_by_step(prune, seed, scale, nsamp, size, expand_pull):
    g, og1, R0, batch = _dynamic_case(seed, scale, nsamp, size)
    _check_dfp_step_by_step(g, og1, R0, batch, prune, expand_pull)


@pytest.mark.parametrize("expand_pull", [1 / 16, 0.0, 2.0])
@pytest.mark.parametrize("prune", [1, 0])
def test_dfp_hub_rows_step_by_step(prune, expand_pull):
    """Rows of in-degree above 4096 run the block-per-vertex kernel of the DF / DF-P sweep (the highest
    in-degree class under the default thresholds): two planted in-hubs (about 19 K and 7 K sources) whose
    in-rows the batch changes, flags exact and ranks to 1e-12 against the oracle, step by step."""
    n, s, d, extra = planted_hub_case(11)
    g, og1, R0, batch = batch_case(n, s, d, 11, 40, extra=extra)
    assert (og1.indeg > 4096).sum() == 2
    _check_dfp_step_by_step(g, og1, R0, batch, prune, expand_pull)


@pytest.mark.parametrize("prune", [1, 0])
def test_dfp_vertex_count_not_a_multiple_of_four(prune):
    """n = 4099: the frontier listing reads the flags four at a time and the last three vertices separately;
    with the listed form forced on and off, DF / DF-P match the oracle step by step, and so does DT."""
    n = 4099
    s = synth.randint(40000, n, seed=41)
    d = synth.randint(40000, n, seed=42)
    s = np.concatenate([s, np.full(30, n - 1, np.int32), np.full(30, n - 2, np.int32)])
    d = np.concatenate([d, synth.randint(60, n, seed=43)])
    extra = (np.array([n - 1], np.int32), np.array([int(d[-1])], np.int32), np.array([n - 3, n - 1], np.int32),
             np.array([n - 2, 5], np.int32))
    g, og1, R0, batch = batch_case(n, s, d, 12, 20, extra=extra)
    _check_dfp_step_by_step(g, og1, R0, batch, prune, 1 / 16)
    ds, dd, is_, id_, de, ie, dmo, imo = batch
    Ro, sto, dVo, na, rounds = oracle.pagerank_dt(og1, ds, dd, is_, host(R0), del_mask=dmo, ins_mask=imo)
    for expand_list in (-1, 64):
        R, st, dV = g.pagerank_dt(dev(ds), dev(dd), dev(is_), R0, del_mask=de, ins_mask=ie, want_dV=True,
                                  expand_list=expand_list)
        assert np.array_equal(host(dV), dVo) and st.iterations == sto.iterations
        assert np.max(np.abs(host(R) - Ro) / Ro) <= 1e-12


@pytest.mark.parametrize("expand_pull", [1 / 16, 0.0, 2.0])
@pytest.mark.parametrize("prune", [1, 0])
@pytest.mark.parametrize("thr", [[1, 4, 16, 32, 64], [0, 4]])
def test_dfp_lowered_thresholds_step_by_step(thr, prune, expand_pull):
    """Lowered in-degree thresholds put hundreds of rows into the block-per-vertex class (in-degree above
    64, or above 4) and the warp class: DF / DF-P still match the oracle step by step."""
    g, og1, R0, batch = _dynamic_case(3, 12, 50000, 5, thresholds=thr)
    assert (og1.indeg > thr[-1]).sum() >= 80
    _check_dfp_step_by_step(g, og1, R0, batch, prune, expand_pull)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_and_host_loops_give_the_same_bits(precision):
    """The sweep loop runs as one CUDA graph (default) or from the host (time_sweeps=1): Static, DF-P and DT
    return identical ranks, flags and sweep counts either way, in FP64 and in mixed precision."""
    g, og1, R0, (ds, dd, is_, id_, de, ie, dmo, imo) = _dynamic_case(2, 12, 40000, 30)
    Rg, stg = g.pagerank_static(precision=precision)
    Rh, sth = g.pagerank_static(precision=precision, time_sweeps=1)
    assert torch.equal(Rg, Rh) and stg.iterations == sth.iterations and stg.iterations_fp32 == sth.iterations_fp32
    for call in (g.pagerank_dfp, g.pagerank_dt):
        Rg, stg, dVg = call(dev(ds), dev(dd), dev(is_), R0, del_mask=de, ins_mask=ie, want_dV=True,
                            precision=precision)
        Rh, sth, dVh = call(dev(ds), dev(dd), dev(is_), R0, del_mask=de, ins_mask=ie, want_dV=True,
                            precision=precision, time_sweeps=1)
        assert torch.equal(Rg, Rh) and torch.equal(dVg, dVh)
        assert stg.iterations == sth.iterations and stg.iterations_fp32 == sth.iterations_fp32
        assert sth.sweeps_launched >= sth.iterations and stg.sweeps_launched == stg.iterations


@pytest.mark.parametrize("bad", ["nan", "negative", "inf", "sum"])
def test_start_vectors_outside_the_sweeps_domain_are_rejected(bad):
    """R0 (Naive-dynamic) and prev_ranks (DF-P, DT) must be finite, non-negative and sum to at most 4 (the
    exact accumulator's range); anything else is PRDF_EINVAL and the output is left untouched."""
    P = prdf()
    n, s, d = synth.rmat(10, 8000, seed=4)
    g = gpu_graph(n, s, d)
    R0 = synth.uniform(n, seed=9)
    R0 /= R0.sum()
    if bad == "nan":
        R0[17] = np.nan
    elif bad == "negative":
        R0[3] = -1e-12
    elif bad == "inf":
        R0[n - 1] = np.inf
    else:
        R0 *= 4.5
    R0d = dev(R0)
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    with pytest.raises(P.PrdfError) as ex:
        g.pagerank_static(R0=R0d)
    assert ex.value.code == -1
    for call in (g.pagerank_dfp, g.pagerank_dt):
        with pytest.raises(P.PrdfError) as ex:
            call(e, e, e, R0d)
        assert ex.value.code == -1
    # a valid vector still works after the rejections
    R1 = synth.uniform(n, seed=9)
    R, st = g.pagerank_static(R0=dev(R1 / R1.sum()))
    assert st.converged


def test_dfp_error_against_static_reference():
    g, og1, R0, (ds, dd, is_, id_, de, ie, dmo, imo) = _dynamic_case(4, 14, 1 << 18, 10)
    R, st, _ = g.pagerank_dfp(dev(ds), dev(dd), dev(is_), R0, del_mask=de, ins_mask=ie)
    ref, _ = oracle.static_ref(og1)
    err = np.abs(host(R) - ref).sum()
    assert err <= 0.85 / 0.15 * 1e-6
    # Static stopped at L-inf 1e-10 is itself only within ~alpha/(1-alpha)*tau per vertex of the reference;
    # the GPU's Static error equals the oracle's Static error
    Rs, _ = g.pagerank_static()
    Rso, _ = oracle.pagerank_static(og1)
    assert abs(np.abs(host(Rs) - ref).sum() - np.abs(Rso - ref).sum()) <= 1e-12


def test_dfp_empty_batch_is_identity():
    n, s, d = synth.rmat(10, 12000, seed=5)
    g = gpu_graph(n, s, d)
    R0o, _ = oracle.pagerank_static(oracle.graph(n, s, d))
    R0 = dev(R0o)
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    R, st, dV = g.pagerank_dfp(e, e, e, R0, want_dV=True)
    assert st.iterations == 1 and st.affected_initial == 0
    assert int(dV.sum()) == 0
    # ranks are held as R/|out| on the device: the round trip costs at most one rounding each way
    assert float(((R - R0).abs() / R0).max()) <= 4.5e-16


def test_dfp_all_affected_df_equals_naive_dynamic():
    n, s, d = synth.rmat(11, 30000, seed=8)
    g = gpu_graph(n, s, d)
    og = oracle.graph(n, s, d)
    R0 = synth.uniform(n, seed=5)
    R0 /= R0.sum()
    allv = torch.arange(n, dtype=torch.int32, device="cuda")
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    R, st, _ = g.pagerank_dfp(e, e, allv, dev(R0), prune=0, tau_f=-1.0)
    Rn, stn = oracle.pagerank_static(og, R0=R0)
    assert st.iterations == stn.iterations
    assert np.max(np.abs(host(R) - Rn)) <= 1e-13


# ------------------------------------------------------ Dynamic Traversal ----

@pytest.mark.parametrize("seed,scale,nsamp,size", [(1, 8, 3000, 20), (5, 12, 3000, 8), (6, 12, 50000, 5),
                                                   (7, 14, 20000, 40)])
@pytest.mark.parametrize("expand_list", [-1, 64])
def test_dt_matches_oracle(seed, scale, nsamp, size, expand_list):
    """Closure bit-exact (sparse graphs leave unreachable vertices out), same sweep count, ranks to 1e-12; with
    closure rounds of at most 64 frontier vertices expanded from a list or not."""
    g, og1, R0, (ds, dd, is_, id_, de, ie, dmo, imo) = _dynamic_case(seed, scale, nsamp, size)
    R, st, dV = g.pagerank_dt(dev(ds), dev(dd), dev(is_), R0, del_mask=de, ins_mask=ie, want_dV=True,
                              expand_list=expand_list)
    Ro, sto, dVo, na, rounds = oracle.pagerank_dt(og1, ds, dd, is_, host(R0), del_mask=dmo, ins_mask=imo)
    assert np.array_equal(host(dV), dVo)
    assert st.affected_initial == na
    assert st.iterations == sto.iterations and st.converged
    assert np.max(np.abs(host(R) - Ro) / Ro) <= 1e-12
    unaffected = dVo == 0
    if unaffected.any():  # unaffected vertices keep R^{t-1} up to the x = R/|out| round trip
        r0 = host(R0)[unaffected]
        assert np.max(np.abs(host(R)[unaffected] - r0) / r0) <= 4.5e-16


def test_dt_empty_batch_is_identity():
    n, s, d = synth.rmat(10, 12000, seed=5)
    g = gpu_graph(n, s, d)
    R0o, _ = oracle.pagerank_static(oracle.graph(n, s, d))
    R0 = dev(R0o)
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    R, st, dV = g.pagerank_dt(e, e, e, R0, want_dV=True)
    assert st.iterations == 1 and st.affected_initial == 0
    assert int(dV.sum()) == 0
    assert float(((R - R0).abs() / R0).max()) <= 4.5e-16


def test_module_level_entry_points():
    """prdf.static / prdf.dfp / prdf.dt are the Graph methods of the same job."""
    P = prdf()
    n, s, d = synth.rmat(9, 4000, seed=3)
    g = gpu_graph(n, s, d)
    R1, st1 = P.static(g)
    R2, st2 = g.pagerank_static()
    assert torch.equal(R1, R2) and st1.iterations == st2.iterations
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    for call in (P.dfp, P.dt):
        R, st, _ = call(g, e, e, e, R1)
        assert st.iterations == 1 and float(((R - R1).abs() / R1).max()) <= 4.5e-16


def test_autotune_keeps_ranks_bit_identical():
    """The tuner only changes kernel shapes and the vertex numbering; exact accumulation keeps every bit."""
    n, s, d = synth.rmat(13, 150000, seed=12)
    g = gpu_graph(n, s, d)
    R0, st0 = g.pagerank_static()
    idx, ms = g.autotune(sweeps=3)
    assert 0 <= idx < 8 and ms > 0
    R1, st1 = g.pagerank_static()
    assert torch.equal(R0, R1) and st0.iterations == st1.iterations
