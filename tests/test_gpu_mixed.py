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
from helpers import adversarial_edges, dev, host

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
