"""Pins of the oracle's Chebyshev filter (Algorithm 3) against the closed form (Eqs. (3)-(5)).

The three-term recurrence must equal T_m((x-c)/e) / T_m((a0-c)/e) applied to
exact eigenvectors of graphs whose spectra are known in closed form.  T_m is
evaluated independently with numpy's Chebyshev series.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

import synth
from oracle import chebyshev_filter, filter_polynomial, laplacian_csr


def closed_form(lam, m, a, b, a0):
    c, e = (a + b) / 2, (b - a) / 2
    coef = np.zeros(m + 1)
    coef[m] = 1.0
    return npcheb.chebval((np.asarray(lam) - c) / e, coef) / npcheb.chebval((a0 - c) / e, coef)


def cycle_modes(n):
    i = np.arange(n)
    lams, vecs = [], []
    for j in range(n // 2 + 1):
        lam = 1.0 - math.cos(2 * math.pi * j / n)
        lams.append(lam)
        vecs.append(np.cos(2 * math.pi * j * i / n))
        if 0 < j < n / 2:
            lams.append(lam)
            vecs.append(np.sin(2 * math.pi * j * i / n))
    V = np.stack(vecs, 1)
    return np.array(lams), V / np.linalg.norm(V, axis=0)


def path_modes(n):
    # v_j(i) = sqrt(d_i) cos(pi j i / (n-1)), lambda_j = 1 - cos(pi j / (n-1))
    i = np.arange(n)
    d = np.where((i == 0) | (i == n - 1), 1.0, 2.0)
    lams = 1.0 - np.cos(np.pi * np.arange(n) / (n - 1))
    V = np.sqrt(d)[:, None] * np.cos(np.pi * np.outer(i, np.arange(n)) / (n - 1))
    return lams, V / np.linalg.norm(V, axis=0)


@pytest.mark.parametrize("n", [64, 101])
def test_cycle_modes_are_eigenvectors(n):
    g = synth.cycle_edges(n)
    A = laplacian_csr(g.n, g.src, g.dst).scipy()
    lam, V = cycle_modes(n)
    assert np.abs(A @ V - V * lam).max() < 1e-13


@pytest.mark.parametrize("n", [50, 97])
def test_path_modes_are_eigenvectors(n):
    g = synth.path_edges(n)
    A = laplacian_csr(g.n, g.src, g.dst).scipy()
    lam, V = path_modes(n)
    assert np.abs(A @ V - V * lam).max() < 1e-13


@pytest.mark.parametrize("m,a", [(1, 0.3), (2, 0.3), (11, 0.3), (11, 0.002), (15, 0.2), (15, 0.5), (13, 1.2)])
def test_filter_on_cycle_modes(m, a):
    n = 120
    g = synth.cycle_edges(n)
    A = laplacian_csr(g.n, g.src, g.dst).scipy()
    lam, V = cycle_modes(n)
    out = chebyshev_filter(A, V, m, a, 2.0, 0.0)
    p = closed_form(lam, m, a, 2.0, 0.0)
    scale = max(1.0, np.abs(p).max())
    assert np.abs(out - V * p).max() < 1e-12 * scale
    # p(a0) = 1 and |p| <= |1/T_m(l(a0))| on the damped interval
    assert abs(closed_form([0.0], m, a, 2.0, 0.0)[0] - 1.0) < 1e-14


@pytest.mark.parametrize("m,a", [(11, 0.05), (15, 0.3)])
def test_filter_on_path_modes(m, a):
    n = 80
    g = synth.path_edges(n)
    A = laplacian_csr(g.n, g.src, g.dst).scipy()
    lam, V = path_modes(n)
    out = chebyshev_filter(A, V, m, a, 2.0, 0.0)
    p = closed_form(lam, m, a, 2.0, 0.0)
    assert np.abs(out - V * p).max() < 1e-12 * max(1.0, np.abs(p).max())


def test_filter_on_hypercube_eigenspaces():
    d = 6
    g = synth.hypercube_edges(d)
    A = laplacian_csr(g.n, g.src, g.dst).scipy()
    ev, U = np.linalg.eigh(A.toarray())
    # spectrum 2i/d with multiplicity C(d, i)
    expect = np.sort(np.concatenate([[2 * i / d] * math.comb(d, i) for i in range(d + 1)]))
    assert np.abs(ev - expect).max() < 1e-13
    X = synth.gaussian_block(g.n, 4, 7)
    out = chebyshev_filter(A, X, 9, 0.4, 2.0, 0.0)
    ref = U @ (closed_form(ev, 9, 0.4, 2.0, 0.0)[:, None] * (U.T @ X))
    assert np.abs(out - ref).max() < 1e-11 * np.abs(ref).max()


def test_oracle_closed_form_matches_numpy_chebyshev():
    lam = np.linspace(0, 2, 41)
    for m in (1, 4, 11, 15):
        np.testing.assert_allclose(filter_polynomial(lam, m, 0.25, 2.0, 0.0),
                                   closed_form(lam, m, 0.25, 2.0, 0.0), rtol=1e-11, atol=1e-13)


def test_planted_mistake_is_caught():
    """A recurrence without the -sigma*sigma1*V term must fail the closed-form pin."""
    n, m, a = 60, 7, 0.3
    g = synth.cycle_edges(n)
    A = laplacian_csr(g.n, g.src, g.dst).scipy()
    lam, V = cycle_modes(n)
    c, e = (a + 2.0) / 2, (2.0 - a) / 2
    sigma = e / (0.0 - c)
    tau = 2 / sigma
    U = (A @ V - c * V) * (sigma / e)
    for _ in range(2, m + 1):
        s1 = 1 / (tau - sigma)
        U, sigma = (A @ U - c * U) * (2 * s1 / e), s1   # dropped term
    p = closed_form(lam, m, a, 2.0, 0.0)
    assert np.abs(U - V * p).max() > 1e-3
