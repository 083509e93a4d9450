"""The second workload family on the GPU: the MAWI stand-in (connected power-law graph with
hubs longer than the SpMM segment length and a degree-1 majority) against the oracle's solve
with trajectory parity, and the degree-corrected SBM stand-ins of the Graph Challenge
categories (k = 64 eigenpairs of 100,000-node graphs) against scipy's Lanczos eigensolver,
with their planted partitions recovered by the GPU spectral clustering."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import oracle
import synth
from gpu_util import device_csr, gaussian_v0, oracle_csr, residuals, to_np
from oracle import cluster

pytestmark = pytest.mark.gpu
TOL = 1e-8


@pytest.fixture(scope="module")
def H():
    import paper_2212_04443_gb300 as P
    return P.Handle()


@pytest.mark.parametrize("precision", [0, 1])
def test_powerlaw_matches_oracle(H, precision):
    w = synth.workload("mawi18m@30000")
    g = w["graph"]
    k, b, m, act = 8, 8, 15, 64
    L = oracle_csr(g)
    assert L.degree.max() > 1024                      # hub rows take the segment path
    A = device_csr(H, g)
    ev, V, info = H.solve(A, k, b, m, act, TOL, v_init=gaussian_v0(g.n, b, 0),
                          precision=precision, record_history=True)
    hist = H.history()
    r = oracle.bchdav(L.scipy(), k, b, m, act, TOL, V_init=synth.gaussian_block(g.n, b, 0))
    assert info.status == 0 and r.converged
    ev, V = to_np(ev), to_np(V)
    assert residuals(L.scipy(), ev, V).max() <= TOL * 1.0001
    assert np.abs(ev - r.evals).max() <= 1e-10
    if precision == 0:
        assert info.iters == r.iters
        assert [h.k_c for h in hist] == [h["k_c"] for h in r.history]
    else:
        assert abs(info.iters - r.iters) <= 2


@pytest.mark.parametrize("cat", ["lbolbsv", "hbohbsv"])
def test_dcsbm_matches_lanczos_and_recovers_blocks(H, cat):
    w = synth.workload(f"dcsbm5m_{cat}@100000")
    g = w["graph"]
    k, b, m, act = w["k"], w["b"], w["m"], w["act_max"]
    A = device_csr(H, g)
    ev, V, info = H.solve(A, k, b, m, act, TOL, v_init=gaussian_v0(g.n, b, 0), precision=1)
    assert info.status == 0
    L = oracle_csr(g)
    ev_np = to_np(ev)
    assert residuals(L.scipy(), ev_np, to_np(V)).max() <= TOL * 1.0001
    ref = np.sort(2 - sla.eigsh(2 * sp.identity(g.n) - L.scipy(), k=k, which="LA", tol=1e-12,
                                return_eigenvectors=False))
    assert np.abs(ev_np - ref).max() <= 1e-9
    lab, _, _, _ = H.spectral_cluster(V, 64, synth.kmeans_first(g.n, 0))
    ari = cluster.adjusted_rand_index(to_np(lab), g.labels)
    assert ari >= (0.999 if cat == "lbolbsv" else 0.95), ari
