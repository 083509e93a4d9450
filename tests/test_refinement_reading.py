"""The readings behind the small Step 9 route (csrc/eigs.cu), checked in float64 numpy.

The route refines a float32 eigendecomposition X of H by the iteration of Ogita and Aishima
(2018): R = I - X^T X, S = X^T H X, lam_j = s_jj / (1 - r_jj), E_ij = (s_ij + lam_j r_ij) /
(lam_j - lam_i) for pairs separated by more than delta = 2 (||S - diag lam|| + ||H|| ||R||) and
r_ij / 2 otherwise, X <- X + X E.  Two readings of that iteration are the route's own:

* for i < j only E_ij comes from the formula and E_ji = r_ij - E_ij, so that E + E^T = R to
  rounding and X stays orthonormal to float64 accuracy even where a small gap makes E_ij
  ill-conditioned (taking both from the formula loses orthogonality as eps ||H|| / gap);
* pairs left inside a cluster are accepted only when their coupling |s_ij| is at the level a
  backward-stable solver leaves: an exactly repeated eigenvalue passes (any orthonormal basis
  of its space is right), distinct eigenvalues closer than float32 resolves stay coupled at
  about their gap and are handed to another eigensolver.

Matrices: Q diag(d) Q^T with known spectra (no GPU)."""
import numpy as np
import pytest

import synth


def refine(H, X, pair, maxit=6, stop=1e-8):
    n = H.shape[0]
    nH = np.linalg.norm(H)
    for _ in range(maxit):
        G = X.T @ X
        R = np.eye(n) - G
        S = X.T @ (H @ X)
        lam = np.diag(S) / np.diag(G)
        delta = 2 * (np.linalg.norm(S - np.diag(lam)) + nH * np.linalg.norm(R))
        gap = lam[None, :] - lam[:, None]                      # lam_j - lam_i
        clus = np.abs(gap) <= delta
        E = np.where(clus, R / 2, (S + lam[None, :] * R) / np.where(clus, 1.0, gap))
        np.fill_diagonal(E, np.diag(R) / 2)
        if pair:
            E = np.triu(E) + np.tril((R - E).T, -1)           # E_ji = r_ij - E_ij, i < j
        off = clus & ~np.eye(n, dtype=bool)
        coupling = np.abs(S[off]).max() / nH if off.any() else 0.0
        emax = np.abs(E).max()
        X = X + X @ E
        if emax <= stop:
            break
    return X, lam, emax, coupling


def spectrum_matrix(d, seed):
    n = d.size
    Q = np.linalg.qr(synth.gaussian_block(n, n, seed))[0]
    H = (Q * d) @ Q.T
    return (H + H.T) / 2


def float32_start(H):
    _, Z = np.linalg.eigh(H.astype(np.float32))
    return Z.astype(np.float64)


@pytest.mark.parametrize("gap", [1e-5, 1e-4])
def test_pairing_keeps_orthogonality_where_the_formula_alone_loses_it(gap):
    n = 40
    d = np.concatenate([0.3 + gap * np.arange(6), np.linspace(0.5, 1.8, n - 6)])
    H = spectrum_matrix(d, 3)
    X0 = float32_start(H)
    Xp, lam_p, emax_p, _ = refine(H, X0, pair=True)
    Xf, lam_f, emax_f, _ = refine(H, X0, pair=False)
    orth_p = np.abs(Xp.T @ Xp - np.eye(n)).max()
    orth_f = np.abs(Xf.T @ Xf - np.eye(n)).max()
    assert emax_p <= 1e-7
    assert orth_p < 1e-14
    assert orth_f > 20 * orth_p          # eps ||H|| / gap, measured ~1e-13 .. 1e-12
    assert np.abs(np.sort(lam_p) - np.sort(d)).max() < 1e-14
    assert np.abs(H @ Xp - Xp * lam_p).max() < 1e-14


def test_exact_repeats_pass_the_coupling_test():
    n = 32
    d = np.concatenate([np.zeros(8), np.full(6, 0.5), np.linspace(0.7, 2.0, n - 14)])
    H = spectrum_matrix(d, 5)
    X, lam, emax, coupling = refine(H, float32_start(H), pair=True)
    assert emax <= 1e-7
    assert coupling <= 4e-15 * n
    assert np.abs(X.T @ X - np.eye(n)).max() < 1e-14
    assert np.abs(np.sort(lam) - np.sort(d)).max() < 1e-14


def test_distinct_eigenvalues_below_float32_resolution_stay_coupled():
    """A chain 1e-9 apart: float32 cannot tell them apart, the iteration treats the chain as one
    cluster and leaves it mixed -- coupled far above the acceptance level, so the route hands the
    matrix on instead of returning Rayleigh quotients wrong by about the gap."""
    n = 32
    d = np.concatenate([0.3 + 1e-9 * np.arange(5), np.linspace(0.5, 1.8, n - 5)])
    H = spectrum_matrix(d, 7)
    X, lam, emax, coupling = refine(H, float32_start(H), pair=True)
    assert coupling > 4e-15 * n
