"""Pins of the combinatorial Laplacian (oracle/laplacian.py, kind="combinatorial"), the k-step
Lanczos bound estimator (oracle/lanczos.py) and Algorithm 2 run with estimated bounds:
closed-form spectra, the relation to Eq. (1), the Lanczos relation, exactness after N steps,
bounds that enclose known spectra, and a solve against dense brute force."""
from math import comb

import numpy as np
import pytest

import oracle
import synth
from oracle import lanczos as LZ


def _comb(g):
    return oracle.laplacian_csr(g.n, g.src, g.dst, kind="combinatorial")


@pytest.mark.parametrize("n", [5, 8, 13])
def test_combinatorial_cycle_and_path(n):
    w = np.linalg.eigvalsh(_comb(synth.cycle_edges(n)).dense())
    want = np.sort(2 - 2 * np.cos(2 * np.pi * np.arange(n) / n))
    assert np.allclose(w, want, atol=1e-12)
    w = np.linalg.eigvalsh(_comb(synth.path_edges(n)).dense())
    assert np.allclose(w, np.sort(2 - 2 * np.cos(np.pi * np.arange(n) / n)), atol=1e-12)


def test_combinatorial_complete_bipartite_hypercube():
    w = np.linalg.eigvalsh(_comb(synth.complete_edges(7)).dense())
    assert np.allclose(w, [0] + [7] * 6, atol=1e-12)
    w = np.linalg.eigvalsh(_comb(synth.complete_bipartite_edges(3, 5)).dense())
    assert np.allclose(w, sorted([0] + [3] * 4 + [5] * 2 + [8]), atol=1e-12)
    d = 5
    w = np.linalg.eigvalsh(_comb(synth.hypercube_edges(d)).dense())
    want = np.sort(np.concatenate([[2.0 * i] * comb(d, i) for i in range(d + 1)]))
    assert np.allclose(w, want, atol=1e-12)


def test_combinatorial_entries_and_relation_to_eq1():
    g = synth.disjoint_union(synth.star_edges(4), synth.path_edges(1))   # node 5 isolated
    L = _comb(g).dense()
    assert L[0, 0] == 4 and np.all(L[0, 1:5] == -1) and L[1, 1] == 1
    assert np.all(L[5] == 0)                         # isolated node: zero row, zero diagonal
    assert np.allclose(L.sum(axis=1), 0)
    h = synth.sbm_edges(300, 3, d_in=8, d_out=1, seed=3)
    Lc, Ln = _comb(h), oracle.laplacian_csr(h.n, h.src, h.dst)
    assert np.array_equal(Lc.colidx, Ln.colidx) and np.array_equal(Lc.rowptr, Ln.rowptr)
    s = np.sqrt(Lc.degree.astype(float))
    assert np.allclose(s[:, None] * Ln.dense() * s[None, :], Lc.dense(), atol=1e-12)


def _sbm_comb(n=2000):
    return _comb(synth.sbm_edges(n, 5, d_in=12, d_out=2, seed=4)).scipy()


def test_lanczos_relation_and_orthogonality():
    A = _sbm_comb()
    k = 20
    alpha, beta, V = LZ.lanczos(A, LZ.start_vector(A.shape[0], 7), k)
    T = LZ.tridiagonal(alpha, beta)
    Vk = V[:, :k]
    R = A @ Vk - Vk @ T
    R[:, -1] -= beta[-1] * V[:, k]
    assert np.linalg.norm(R) <= 1e-12 * np.linalg.norm(T)
    assert np.abs(V[:, :10].T @ V[:, :10] - np.eye(10)).max() < 1e-10
    assert abs(np.linalg.norm(LZ.start_vector(A.shape[0], 7)) - 1) < 1e-15


def test_lanczos_exact_after_n_steps_and_invariant_subspace():
    d = np.array([-3.0, -1.0, 0.5, 1.0, 2.0, 2.5, 4.0, 7.0, 9.0, 11.0])
    A = np.diag(d)
    alpha, beta, _ = LZ.lanczos(A, LZ.start_vector(10, 1), 10)
    assert np.allclose(np.linalg.eigvalsh(LZ.tridiagonal(alpha, beta)), d, atol=1e-10)
    assert abs(beta[-1]) < 1e-10
    alpha, beta, _ = LZ.lanczos(3.0 * np.eye(6), LZ.start_vector(6, 2), 5)
    assert alpha.tolist() == [3.0] and beta.tolist() == [0.0]   # stops after one step
    lo, hi, _, _ = LZ.bounds(3.0 * np.eye(6), 5, 2)
    assert lo == hi == 3.0


@pytest.mark.parametrize("kind", ["normalized", "combinatorial"])
@pytest.mark.parametrize("graph", ["cycle", "hypercube", "complete", "sbm"])
def test_bounds_enclose_the_spectrum(kind, graph):
    g = {"cycle": synth.cycle_edges(101), "hypercube": synth.hypercube_edges(7),
         "complete": synth.complete_edges(40),
         "sbm": synth.sbm_edges(1500, 4, d_in=10, d_out=2, seed=5)}[graph]
    L = oracle.laplacian_csr(g.n, g.src, g.dst, kind=kind)
    w = np.linalg.eigvalsh(L.dense())
    for k in (10, 20):
        lo, hi, _, _ = LZ.bounds(L.scipy(), k, 11)
        assert hi >= w[-1] - 1e-12                   # a bound from above of the largest
        assert w[0] - 1e-12 <= lo <= w[-1]           # a Ritz value: inside the spectrum


def test_solve_with_lanczos_bounds_matches_brute_force():
    g = synth.sbm_edges(600, 4, d_in=14, d_out=1.5, seed=6)
    L = _comb(g)
    lo, hi, _, _ = LZ.bounds(L.scipy(), 20, 0)
    w = np.linalg.eigvalsh(L.dense())
    r = oracle.bchdav(L.scipy(), 6, 6, 11, 36, 1e-8, bounds=(lo, hi))
    assert r.converged
    assert np.allclose(r.evals, w[:6], atol=1e-8 * hi)
    assert oracle.relative_residuals(L.scipy(), r.evals, r.evecs).max() <= 1e-8 * 1.0001
