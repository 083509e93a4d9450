"""Failure paths of bchdav_solve made on the host, none of which faults the GPU: a non-finite
initial block (BCHDAV_ERR_NONFINITE before any iteration) and a workspace allocation that fails
(BCHDAV_ERR_OOM, forced by the handle's workspace cap).  After each failure the same handle
solves the same problem correctly."""
import numpy as np
import pytest

import synth
from gpu_util import device_csr, gaussian_v0, oracle_csr, residuals, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-8


@pytest.fixture(scope="module")
def problem():
    g = synth.sbm_edges(4000, 6, d_in=10, d_out=1.5, seed=12)
    return g, 6, 6, 11, 30


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_nonfinite_v_init(problem, bad):
    import paper_2212_04443_gb300 as P
    g, k, b, m, act = problem
    H = P.Handle()
    A = device_csr(H, g)
    V0 = gaussian_v0(g.n, b)
    V0[1234, 3] = bad
    with pytest.raises(P.BchdavError) as ei:
        H.solve(A, k, b, m, act, TOL, v_init=V0)
    assert ei.value.status == -5
    assert "v_init" in str(ei.value)
    # the same handle, a finite block: a normal solve
    ev, V, info = H.solve(A, k, b, m, act, TOL, v_init=gaussian_v0(g.n, b))
    assert info.status == 0
    assert residuals(oracle_csr(g).scipy(), to_np(ev), to_np(V)).max() <= TOL * 1.0001


def test_allocation_failure_then_recovery(problem):
    import paper_2212_04443_gb300 as P
    g, k, b, m, act = problem
    H = P.Handle()
    A = device_csr(H, g)
    V0 = gaussian_v0(g.n, b)
    ev0, V0out, info0 = H.solve(A, k, b, m, act, TOL, v_init=V0)
    assert info0.status == 0
    need = H.workspace_bytes()
    assert need > 0
    # a fresh handle capped below what the solve needs: the workspace cannot be allocated
    H2 = P.Handle()
    H2.set_memory_limit(need // 4)
    with pytest.raises(P.BchdavError) as ei:
        H2.solve(A, k, b, m, act, TOL, v_init=V0)
    assert ei.value.status == -3
    assert H2.workspace_bytes() <= need // 4
    # lift the cap: the same handle now solves, with the result of the uncapped handle
    H2.set_memory_limit(0)
    ev, V, info = H2.solve(A, k, b, m, act, TOL, v_init=V0)
    assert info.status == 0
    assert np.array_equal(to_np(ev), to_np(ev0)) and np.array_equal(to_np(V), to_np(V0out))


def test_allocation_failure_keeps_held_workspace(problem):
    """A larger problem on a handle whose cap only fits the smaller one fails with
    BCHDAV_ERR_OOM without freeing what the handle holds; the smaller problem still solves."""
    import paper_2212_04443_gb300 as P
    g, k, b, m, act = problem
    H = P.Handle()
    A = device_csr(H, g)
    V0 = gaussian_v0(g.n, b)
    ev0, _, info0 = H.solve(A, k, b, m, act, TOL, v_init=V0)
    held = H.workspace_bytes()
    big = synth.sbm_edges(60000, 6, d_in=10, d_out=1.5, seed=12)
    Ab = device_csr(H, big)
    H.set_memory_limit(held)
    with pytest.raises(P.BchdavError) as ei:
        H.solve(Ab, k, b, m, act, TOL, v_init=gaussian_v0(big.n, b))
    assert ei.value.status == -3
    assert H.workspace_bytes() <= held
    ev, _, info = H.solve(A, k, b, m, act, TOL, v_init=V0)
    assert info.status == 0 and np.array_equal(to_np(ev), to_np(ev0))
