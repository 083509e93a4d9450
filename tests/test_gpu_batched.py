"""Many independent solves in one call (bchdav_solve_batched) against the oracle's brute
force and against one-at-a-time solves of the same graphs."""
import numpy as np
import pytest

import synth
from gpu_util import device_csr, oracle_csr, residuals, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-8


@pytest.fixture(scope="module")
def H():
    import paper_2212_04443_gb300 as P
    return P.Handle()


def _batch(n_graphs, seed):
    """Uneven SBM graphs shaped like the batched workload (log-uniform sizes, c in [4, 32],
    intra-degree 12, inter-degree 1.5), scaled down so that brute force stays cheap."""
    g = synth.rng(seed)
    ns = np.floor(np.exp(g.uniform(np.log(600), np.log(2500), n_graphs))).astype(int)
    cs = g.integers(4, 13, n_graphs)
    return [synth.sbm_edges(int(ns[i]), int(cs[i]), d_in=12.0, d_out=1.5, seed=500 + i)
            for i in range(n_graphs)], cs


@pytest.mark.parametrize("workers", [1, 4, 8])
def test_batched_matches_brute_force(H, workers):
    import paper_2212_04443_gb300 as P
    graphs, cs = _batch(12, 3)
    As = [device_csr(H, g) for g in graphs]
    ks = [int(c) for c in cs]
    bs = [min(int(c), 8) for c in cs]
    ms = [11] * len(graphs)
    ev, V, infos, ms_per = H.solve_batched(As, ks, bs, ms, [0] * len(graphs), TOL,
                                           precision=P.PREC_MIXED, seed=9, workers=workers)
    assert all(i.status == 0 for i in infos)
    assert np.all(ms_per > 0)
    for i, g in enumerate(graphs):
        L = oracle_csr(g)
        e, v = to_np(ev[i]), to_np(V[i])
        ref = np.linalg.eigvalsh(L.dense())[:ks[i]]
        assert np.abs(e - ref).max() < 1e-10, i
        assert residuals(L.scipy(), e, v).max() <= TOL * 1.0001
        assert np.abs(v.T @ v - np.eye(ks[i])).max() < 1e-10   # mixed path: 36-bit rotations


def test_batched_equals_single_solves(H):
    """Graph i of a batch is the solve of graph i alone with seed + i."""
    import paper_2212_04443_gb300 as P
    graphs, cs = _batch(6, 4)
    As = [device_csr(H, g) for g in graphs]
    ks = [int(c) for c in cs]
    bs = [min(int(c), 8) for c in cs]
    ev, V, infos, _ = H.solve_batched(As, ks, bs, [11] * 6, [0] * 6, TOL,
                                      precision=P.PREC_FP64, seed=21, workers=3)
    for i in range(6):
        e1, v1, info = H.solve(As[i], ks[i], bs[i], 11, 0, TOL, precision=P.PREC_FP64,
                               seed=21 + i)
        # the workers' eigensolver runs on one block: its sums may round differently
        assert abs(infos[i].iters - info.iters) <= 1
        assert np.abs(to_np(ev[i]) - to_np(e1)).max() < 1e-10


def test_batched_reports_failing_graph(H):
    import paper_2212_04443_gb300 as P
    graphs, cs = _batch(3, 5)
    As = [device_csr(H, g) for g in graphs]
    ks = [int(c) for c in cs]
    ks[1] = graphs[1].n + 5                       # k > N: invalid for graph 1 only
    with pytest.raises(P.BchdavError) as ei:
        H.solve_batched(As, ks, [4, 4, 4], [11] * 3, [0] * 3, TOL, workers=2)
    assert ei.value.status == -1
    assert "graph 1" in str(ei.value)
