"""Pins of the oracle's Laplacian (Eq. (1)) against hand-computed entries and invariants."""
import math

import numpy as np
import pytest

import synth
from oracle import laplacian_csr

pytestmark = pytest.mark.filterwarnings("ignore")


def test_path3_hand_computed():
    # P3: degrees 1, 2, 1 -> off-diagonal -1/sqrt(1*2)
    L = laplacian_csr(3, [0, 1], [1, 2])
    s = 1.0 / math.sqrt(2.0)
    expect = np.array([[1.0, -s, 0.0], [-s, 1.0, -s], [0.0, -s, 1.0]])
    assert np.array_equal(L.rowptr, [0, 2, 5, 7])
    assert np.array_equal(L.colidx, [0, 1, 0, 1, 2, 1, 2])
    np.testing.assert_allclose(L.dense(), expect, rtol=0, atol=1e-16)


def test_complete_bipartite_values():
    # K_{2,3}: part-a degree 3, part-b degree 2 -> every edge value -1/sqrt(6)
    g = synth.complete_bipartite_edges(2, 3)
    L = laplacian_csr(g.n, g.src, g.dst)
    D = L.dense()
    off = D[:2, 2:]
    np.testing.assert_allclose(off, -1.0 / math.sqrt(6.0), rtol=1e-15)
    assert np.all(D[:2, :2] == np.eye(2)) and np.all(D[2:, 2:] == np.eye(3))


def test_star_values():
    g = synth.star_edges(7)
    D = laplacian_csr(g.n, g.src, g.dst).dense()
    np.testing.assert_allclose(D[0, 1:], -1.0 / math.sqrt(7.0), rtol=1e-15)
    np.testing.assert_allclose(np.diag(D), 1.0)


def test_selfloops_duplicates_isolated():
    # edges with both orientations, repeats and a self loop; node 4 isolated
    src = [0, 1, 1, 2, 2, 3, 0]
    dst = [1, 0, 2, 1, 2, 2, 1]
    L = laplacian_csr(5, src, dst)
    ref = laplacian_csr(5, [0, 1, 2], [1, 2, 3])
    assert np.array_equal(L.rowptr, ref.rowptr)
    assert np.array_equal(L.colidx, ref.colidx)
    assert np.array_equal(L.val, ref.val)
    # isolated node: a lone diagonal 1
    assert L.rowptr[5] - L.rowptr[4] == 1 and L.colidx[-1] == 4 and L.val[-1] == 1.0
    assert list(L.degree) == [1, 2, 2, 1, 0]


def test_canonical_order_and_symmetry():
    g = synth.sbm_edges(500, 5, d_in=6, d_out=1, seed=11)
    L = laplacian_csr(g.n, g.src, g.dst)
    for i in range(g.n):
        row = L.colidx[L.rowptr[i]:L.rowptr[i + 1]]
        assert np.all(np.diff(row) > 0)
        assert i in row
    S = L.scipy()
    assert abs(S - S.T).max() == 0.0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_spectrum_in_0_2_and_null_vector(seed):
    g = synth.sbm_edges(150, 3, d_in=5, d_out=1, seed=seed)
    L = laplacian_csr(g.n, g.src, g.dst)
    ev = np.linalg.eigvalsh(L.dense())
    assert ev.min() > -1e-12 and ev.max() < 2 + 1e-12
    # D^{1/2} 1 lies in the null space (rows with degree 0 excluded)
    u = np.sqrt(L.degree.astype(float))
    assert np.abs(L.scipy() @ u).max() < 1e-13


def test_bipartite_has_eigenvalue_two():
    g = synth.cycle_edges(10)  # even cycle is bipartite
    L = laplacian_csr(g.n, g.src, g.dst)
    ev = np.linalg.eigvalsh(L.dense())
    assert abs(ev.max() - 2.0) < 1e-14
