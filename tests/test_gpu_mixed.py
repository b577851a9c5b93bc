"""Mixed precision (FP32 ranks with compensated sums, then FP64 refinement
sweeps): the final ranks meet the same FP64 parity target as the FP64 path,
L-inf <= 1e-8 against the FP64 oracle, and the FP32 stage alone stays within
FP32 accuracy of the oracle. The error against the oracle is checked for
every result."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import adversarial_edges, dev, dynamic_case, host

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


@pytest.mark.parametrize("name,n,src,dst", adversarial_edges())
def test_mixed_adversarial(name, n, src, dst):
    g = gpu_graph(n, src, dst)
    R, st = g.pagerank_static(precision=prdf().PRDF_FP32_REFINE)
    Ro, _ = oracle.pagerank_static(oracle.graph(n, src, dst))
    assert np.max(np.abs(host(R) - Ro)) <= 1e-8
    assert st.converged


def test_mixed_rmat_scale16_config():
    n, s, d = synth.rmat(16, 1 << 20, seed=1)
    g = gpu_graph(n, s, d)
    og = oracle.graph(n, s, d)
    R, st = g.pagerank_static(precision=prdf().PRDF_FP32_REFINE)
    ref, _ = oracle.static_ref(og)
    Ro, sto = oracle.pagerank_static(og)
    err = np.max(np.abs(host(R) - ref))
    assert err <= 1e-8, err
    # as close to the fixed point as the FP64 path: within the tail bound of the same stop rule
    assert err <= 2 * np.max(np.abs(Ro - ref)) + 1e-12
    assert st.converged and 0 < st.iterations_fp32 < st.iterations
    # the FP64 stage needs far fewer sweeps than a from-scratch FP64 solve
    assert st.iterations - st.iterations_fp32 < sto.iterations // 2


def test_fp32_stage_accuracy_and_stop_rule():
    """tol = 1 stops the FP64 stage after one sweep: the result is the FP32
    stage's, one FP64 sweep later. The stop rule max|dR| <= rel * max R bounds
    the L-inf error by the Jacobi tail alpha/(1-alpha) * rel * max R, plus FP32
    rounding (a few ulps of max R)."""
    n, s, d = synth.rmat(14, 200000, seed=2)
    g = gpu_graph(n, s, d)
    ref, _ = oracle.static_ref(oracle.graph(n, s, d))
    for rel in (1e-3, 1e-5):
        R, st = g.pagerank_static(precision=prdf().PRDF_FP32_REFINE, tol=1.0, tol_fp32_rel=rel)
        err = np.max(np.abs(host(R) - ref))
        assert err <= (0.85 / 0.15 * rel + 1e-6) * ref.max(), (rel, err, ref.max())
        assert st.iterations == st.iterations_fp32 + 1


def test_mixed_from_previous_ranks():
    n, s, d = synth.rmat(12, 50000, seed=7)
    og = oracle.graph(n, s, d)
    R0 = synth.uniform(n, seed=3)
    R0 /= R0.sum()
    g = gpu_graph(n, s, d)
    R, st = g.pagerank_static(R0=dev(R0), precision=prdf().PRDF_FP32_REFINE)
    ref, _ = oracle.static_ref(og)
    assert np.max(np.abs(host(R) - ref)) <= 1e-8


# ------------------------------------------------- DF-P / DT in mixed precision ----
# FP32 DF-P sweeps (compensated sums, Alg. update's prune and expand tests in FP32) to the relative stop,
# then FP64 DF-P sweeps from their result, with the affected set they left plus every vertex they moved.
# The FP32 stage decides its prune and expand tests at FP32 resolution, so flags are not compared with the
# FP64 oracle; the final ranks are held to the FP64 path's error targets.

ALPHA = 0.85
PRUNE_BOUND = ALPHA / (1 - ALPHA) * 1e-6  # relative error a pruned vertex may keep (tau_p = 1e-6)


def test_mixed_dfp_within_the_prune_bound_of_the_reference():
    """Default tolerances (tau_f = tau_p = 1e-6) on a 2^14-vertex R-MAT: the same L1 bound against the
    oracle's reference Static ranks as FP64 DF-P, and as close to the FP64 oracle DF-P as that bound."""
    g, og1, R0, (ds, dd, is_, id_, de, ie, dmo, imo) = dynamic_case(4, 14, 1 << 18, 10)
    R, st, _ = g.pagerank_dfp(dev(ds), dev(dd), dev(is_), R0, del_mask=de, ins_mask=ie,
                              precision=prdf().PRDF_FP32_REFINE)
    ref, _ = oracle.static_ref(og1)
    Ro, _, _, _ = oracle.pagerank_dfp(og1, ds, dd, is_, host(R0), del_mask=dmo, ins_mask=imo)
    Rm = host(R)
    assert st.converged and st.iterations_fp32 > 0
    assert np.abs(Rm - ref).sum() <= PRUNE_BOUND
    assert np.max(np.abs(Rm - ref) / ref) <= PRUNE_BOUND
    assert np.abs(Rm - Ro).sum() <= PRUNE_BOUND


@pytest.mark.parametrize("prune", [1, 0])
def test_mixed_dfp_tight_tolerances_reach_the_reference(prune):
    """tau_f = tau_p = 1e-13 and tol = 1e-14: DF-P (and DF) in mixed precision reach the reference Static ranks
    to the same 1e-10 L1 as the oracle's own DF-P with these tolerances; the FP32 stage's rounding does not
    survive the FP64 stage."""
    g, og1, R0, (ds, dd, is_, id_, de, ie, dmo, imo) = dynamic_case(5, 12, 40000, 30)
    kw = dict(tau_f=1e-13, tau_p=1e-13, tol=1e-14, prune=prune)
    R, st, _ = g.pagerank_dfp(dev(ds), dev(dd), dev(is_), R0, del_mask=de, ins_mask=ie,
                              precision=prdf().PRDF_FP32_REFINE, **kw)
    ref, _ = oracle.static_ref(og1)
    Ro, _, _, _ = oracle.pagerank_dfp(og1, ds, dd, is_, host(R0), del_mask=dmo, ins_mask=imo, tau_f=1e-13,
                                      tau_p=1e-13, tol=1e-14, prune=bool(prune))
    assert st.converged and 0 < st.iterations_fp32 < st.iterations
    assert np.abs(Ro - ref).sum() <= 1e-10
    assert np.abs(host(R) - ref).sum() <= 1e-10


def test_mixed_dt_matches_the_oracle():
    """Dynamic Traversal in mixed precision: the closure is integer work (bit-exact); the FP64 stage runs Eq. 1
    on it to the same L-inf 1e-10 stop as the oracle, so both lie within alpha/(1-alpha)*tol of the restricted
    fixed point and within twice that of each other."""
    g, og1, R0, (ds, dd, is_, id_, de, ie, dmo, imo) = dynamic_case(6, 12, 50000, 5)
    R, st, dV = g.pagerank_dt(dev(ds), dev(dd), dev(is_), R0, del_mask=de, ins_mask=ie, want_dV=True,
                              precision=prdf().PRDF_FP32_REFINE)
    Ro, sto, dVo, na, _ = oracle.pagerank_dt(og1, ds, dd, is_, host(R0), del_mask=dmo, ins_mask=imo)
    assert np.array_equal(host(dV), dVo) and st.affected_initial == na
    assert st.converged and st.iterations_fp32 > 0
    assert np.max(np.abs(host(R) - Ro)) <= 2 * ALPHA / (1 - ALPHA) * 1e-10
    unaffected = dVo == 0
    if unaffected.any():  # unaffected vertices keep R^{t-1} up to the x = R/|out| round trip
        r0 = host(R0)[unaffected]
        assert np.max(np.abs(host(R)[unaffected] - r0) / r0) <= 4.5e-16


def test_mixed_dfp_empty_batch_is_identity():
    n, s, d = synth.rmat(10, 12000, seed=5)
    g = gpu_graph(n, s, d)
    R0o, _ = oracle.pagerank_static(oracle.graph(n, s, d))
    R0 = dev(R0o)
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    R, st, dV = g.pagerank_dfp(e, e, e, R0, want_dV=True, precision=prdf().PRDF_FP32_REFINE)
    assert st.affected_initial == 0 and int(dV.sum()) == 0
    assert float(((R - R0).abs() / R0).max()) <= 4.5e-16
