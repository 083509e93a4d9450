"""Pins of the oracle's Algorithm 2 against closed-form spectra, brute force and invariants."""
import math

import numpy as np
import pytest
import scipy.sparse.csgraph as csgraph

import synth
from oracle import bchdav, laplacian_csr, relative_residuals

TOL = 1e-8


def solve(g, k, b, m=11, act_max=None, seed=0, **kw):
    L = laplacian_csr(g.n, g.src, g.dst)
    A = L.scipy()
    V0 = synth.gaussian_block(g.n, b, seed)
    r = bchdav(A, k, b, m, act_max, TOL, V_init=V0, **kw)
    return L, A, r


def check_common(A, r, k):
    assert r.converged
    assert r.evals.shape == (k,) and r.evecs.shape == (A.shape[0], k)
    assert np.all(np.diff(r.evals) >= -1e-14)
    assert r.evals.min() > -1e-12 and r.evals.max() < 2 + 1e-12
    assert relative_residuals(A, r.evals, r.evecs).max() <= TOL * 1.0001
    assert np.abs(r.evecs.T @ r.evecs - np.eye(k)).max() < 1e-12


@pytest.mark.parametrize("n,k,b", [(150, 7, 4), (301, 10, 5)])
def test_cycle_closed_form(n, k, b):
    _, A, r = solve(synth.cycle_edges(n), k, b)
    check_common(A, r, k)
    expect = np.sort(1.0 - np.cos(2 * np.pi * np.arange(n) / n))[:k]
    assert np.abs(r.evals - expect).max() < 1e-10


@pytest.mark.parametrize("n,k,b", [(120, 6, 3), (200, 8, 4)])
def test_path_closed_form_values_and_vectors(n, k, b):
    L, A, r = solve(synth.path_edges(n), k, b)
    check_common(A, r, k)
    j = np.arange(k)
    assert np.abs(r.evals - (1.0 - np.cos(np.pi * j / (n - 1)))).max() < 1e-10
    i = np.arange(n)
    d = np.where((i == 0) | (i == n - 1), 1.0, 2.0)
    U = np.sqrt(d)[:, None] * np.cos(np.pi * np.outer(i, j) / (n - 1))
    U /= np.linalg.norm(U, axis=0)
    # simple eigenvalues: vectors agree up to sign
    assert np.abs(np.abs(np.sum(U * r.evecs, 0)) - 1.0).max() < 1e-8


def test_hypercube_closed_form():
    # block size >= multiplicity of 2/d (= d), as block methods need to resolve it
    d = 6
    _, A, r = solve(synth.hypercube_edges(d), 7, 7, act_max=21)
    check_common(A, r, 7)
    expect = np.sort(np.concatenate([[2 * i / d] * math.comb(d, i) for i in range(d + 1)]))[:7]
    assert np.abs(r.evals - expect).max() < 1e-10


def test_complete_graph():
    n = 40
    _, A, r = solve(synth.complete_edges(n), 5, 3, act_max=12)
    check_common(A, r, 5)
    expect = np.array([0.0] + [n / (n - 1)] * 4)
    assert np.abs(r.evals - expect).max() < 1e-10


def test_complete_bipartite():
    a, bb = 9, 14
    _, A, r = solve(synth.complete_bipartite_edges(a, bb), 4, 2, act_max=8)
    check_common(A, r, 4)
    assert np.abs(r.evals - np.array([0.0, 1.0, 1.0, 1.0])).max() < 1e-10


def test_disjoint_union_null_space():
    parts = [synth.cycle_edges(30), synth.path_edges(25), synth.complete_edges(12),
             synth.hypercube_edges(4), synth.star_edges(9)]
    g = synth.disjoint_union(*parts)
    # block size >= zero multiplicity (5)
    L, A, r = solve(g, 6, 5, act_max=15)
    check_common(A, r, 6)
    ncomp, lab = csgraph.connected_components(A, directed=False)
    assert ncomp == 5
    assert np.abs(r.evals[:5]).max() < 1e-10   # zero multiplicity = number of components
    assert r.evals[5] > 1e-3
    # null-space membership: each null vector lies in span{D^{1/2} 1_C}
    sq = np.sqrt(L.degree.astype(float))
    U = np.zeros((g.n, ncomp))
    for c in range(ncomp):
        U[lab == c, c] = sq[lab == c]
    U /= np.linalg.norm(U, axis=0)
    Z = r.evecs[:, :5]
    assert np.abs(Z - U @ (U.T @ Z)).max() < 1e-8


@pytest.mark.parametrize("seed", [21, 22, 23, 24])
def test_dense_brute_force(seed):
    gen = synth.rng(seed)
    n = int(gen.integers(80, 200))
    c = int(gen.integers(2, 5))
    g = synth.sbm_edges(n, c, d_in=8, d_out=1.5, seed=seed)
    L, A, r = solve(g, 8, 4, m=int(gen.integers(5, 13)), act_max=20, seed=seed)
    check_common(A, r, 8)
    ev = np.linalg.eigvalsh(L.dense())
    assert np.abs(r.evals - ev[:8]).max() < 1e-10


def test_connected_null_vector_is_sqrt_degree():
    g = synth.sbm_edges(400, 4, d_in=10, d_out=2, seed=31)
    L, A, r = solve(g, 5, 5, act_max=30)
    check_common(A, r, 5)
    assert abs(r.evals[0]) < 1e-10
    u = np.sqrt(L.degree.astype(float))
    u /= np.linalg.norm(u)
    assert abs(abs(u @ r.evecs[:, 0]) - 1.0) < 1e-10


def test_progressive_filtering_with_exact_initials():
    n, k, b = 160, 4, 2
    g = synth.path_edges(n)
    L = laplacian_csr(g.n, g.src, g.dst)
    A = L.scipy()
    ev, U = np.linalg.eigh(L.dense())
    r = bchdav(A, k, b, 5, 8, TOL, V_init=U[:, :k])
    assert r.converged and r.iters == 2
    assert np.abs(r.evals - ev[:k]).max() < 1e-12


def test_fewer_initials_than_block_uses_random_fill():
    g = synth.cycle_edges(90)
    L = laplacian_csr(g.n, g.src, g.dst)
    A = L.scipy()
    r = bchdav(A, 5, 4, 11, 16, TOL, V_init=synth.gaussian_block(g.n, 1, 3))
    check_common(A, r, 5)
    r2 = bchdav(A, 5, 4, 11, 16, TOL, V_init=None)
    check_common(A, r2, 5)
    assert np.abs(r.evals - r2.evals).max() < 1e-10


def test_itmax_reports_not_converged():
    g = synth.cycle_edges(200)
    L = laplacian_csr(g.n, g.src, g.dst)
    r = bchdav(L.scipy(), 6, 3, 11, 15, TOL, V_init=synth.gaussian_block(g.n, 3, 0), itmax=1)
    assert not r.converged and r.iters == 1


def test_restart_counters_invariant():
    g = synth.sbm_edges(600, 6, d_in=9, d_out=1.5, seed=41)
    _, A, r = solve(g, 12, 4, m=7, act_max=20)
    check_common(A, r, 12)
    for h in r.history:
        assert h["k_sub"] == h["k_c"] - h["e_c"] + h["k_act"]   # k_c + k_act = k_sub (before shift)
        assert h["k_act"] <= 20
