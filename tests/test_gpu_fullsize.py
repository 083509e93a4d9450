"""The solve at the size and in the configuration bench.py times (SBM N = 1,000,000, 100
clusters, k = 100, b = 20, m = 15, act_max = 300, mixed precision, slice products), checked by
properties that hold at any size: every residual recomputed in float64 by scipy at or below the
tolerance, orthonormal eigenvectors, the spectrum inside [0, 2] with lambda_1 = 0 and eigenvector
D^{1/2} 1 (the graph is connected), and the float64 path's eigenvalues within 1e-10."""
import numpy as np
import pytest
import scipy.sparse.csgraph as csgraph

import synth
from gpu_util import device_csr, gaussian_v0, oracle_csr, residuals, to_np

pytestmark = pytest.mark.gpu


def test_bench_workload_properties():
    import paper_2212_04443_gb300 as P
    w = synth.workload("sbm1m")
    g = w["graph"]
    k, b, m, act, tol = w["k"], w["b"], w["m"], w["act_max"], w["tol"]
    H = P.Handle()
    A = device_csr(H, g)
    V0 = gaussian_v0(g.n, b, w["v0_seed"])
    ev, V, info = H.solve(A, k, b, m, act, tol, v_init=V0, precision=P.PREC_MIXED, itmax=200)
    assert info.status == 0
    ev, V = to_np(ev), to_np(V)
    L = oracle_csr(g)
    As = L.scipy()
    assert csgraph.connected_components(As, directed=False)[0] == 1
    assert residuals(As, ev, V).max() <= tol * 1.0001
    assert np.abs(V.T @ V - np.eye(k)).max() < 1e-10
    assert np.all(np.diff(ev) >= -1e-14) and ev[0] > -1e-10 and ev[-1] < 2
    assert abs(ev[0]) < 1e-10
    u = np.sqrt(L.degree.astype(float))
    u /= np.linalg.norm(u)
    assert abs(abs(u @ V[:, 0]) - 1.0) < 1e-10
    ev64, _, info64 = H.solve(A, k, b, m, act, tol, v_init=V0, precision=P.PREC_FP64, itmax=200)
    assert info64.status == 0
    assert np.abs(to_np(ev64) - ev).max() < 1e-10
