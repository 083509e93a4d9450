"""Step 9 for n <= 64 (the small route: a float32 decomposition refined in float64 by the
Ogita-Aishima iteration), through bchdav_eigh, against LAPACK and known spectra.

The route hands the matrix to the Jacobi kernel when its refinement does not settle or leaves a
cluster coupled; every case below must come out right either way.  Sizes cover n = 1, the
smallest cluster shares (n < 16 leaves CTAs without columns), odd and even n and the route's
limit; spectra cover exact repeats, near repeats below the float32 resolution, a zero and a
diagonal matrix, scales near the float64 range ends, wide dynamic range, and the diagonal plus
border shape that Step 15 leaves."""
import numpy as np
import pytest

import synth
from gpu_util import to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import paper_2212_04443_gb300 as P
    return P.Handle()


def eigh(H, S):
    import torch
    D, Y = H.eigh(torch.from_numpy(np.ascontiguousarray(S)).cuda())
    return to_np(D), to_np(Y)


def check(S, D, Y, ref=None, tol=1e-13):
    n = S.shape[0]
    ref = np.linalg.eigvalsh(S) if ref is None else np.sort(ref)
    scale = max(1e-300, np.abs(ref).max(), np.linalg.norm(S, 2))
    assert np.all(np.diff(D) >= 0)
    assert np.abs(D - ref).max() <= tol * scale * max(1, n) ** 0.5
    assert np.abs(Y.T @ Y - np.eye(n)).max() <= tol * max(1, n)
    assert np.abs(S @ Y - Y * D).max() <= tol * scale * max(1, n)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 15, 16, 17, 31, 32, 33, 40, 48, 63, 64])
def test_small_random(H, n):
    rng = synth.rng(1000 + n)
    M = rng.standard_normal((n, n))
    S = (M + M.T) / 2
    D, Y = eigh(H, S)
    check(S, D, Y)


@pytest.mark.parametrize("n", [12, 48, 64])
def test_small_exact_repeats(H, n):
    """Eigenvalues of multiplicity n/4 and n/6: any orthonormal basis of each space is right."""
    Q = np.linalg.qr(synth.gaussian_block(n, n, n))[0]
    a, b = n // 4, n // 6
    d = np.concatenate([np.zeros(a), np.full(b, 0.5), np.linspace(0.6, 2.0, n - a - b)])
    S = (Q * d) @ Q.T
    S = (S + S.T) / 2
    D, Y = eigh(H, S)
    check(S, D, Y, ref=d, tol=1e-13)


@pytest.mark.parametrize("spacing", [1e-13, 1e-9, 1e-6, 1e-4])
def test_small_near_repeats(H, spacing):
    """Chains of eigenvalues closer than float32 resolves (1e-13 .. 1e-6) and one it resolves."""
    n = 48
    Q = np.linalg.qr(synth.gaussian_block(n, n, 31))[0]
    d = np.concatenate([0.3 + spacing * np.arange(10), np.linspace(0.5, 1.8, n - 10)])
    S = (Q * d) @ Q.T
    S = (S + S.T) / 2
    D, Y = eigh(H, S)
    check(S, D, Y, ref=d)


def test_small_zero_and_diagonal(H):
    for n in (1, 7, 40):
        S = np.zeros((n, n))
        D, Y = eigh(H, S)
        assert np.all(D == 0) and np.abs(Y.T @ Y - np.eye(n)).max() == 0
    d = synth.rng(5).uniform(-1, 1, 40)
    S = np.diag(d)
    D, Y = eigh(H, S)
    check(S, D, Y, ref=d)


@pytest.mark.parametrize("scale", [1e-150, 1e-20, 1e20, 1e150])
def test_small_scaled(H, scale):
    n = 40
    M = synth.rng(8).standard_normal((n, n))
    S = scale * (M + M.T) / 2
    D, Y = eigh(H, S)
    check(S, D, Y)


def test_small_wide_dynamic_range(H):
    """Eigenvalues from 1e-12 to 1: float32 sees the small ones as zero, the float64 refinement
    brings them back to float64 accuracy relative to ||H||."""
    n = 32
    Q = np.linalg.qr(synth.gaussian_block(n, n, 3))[0]
    d = np.logspace(-12, 0, n)
    S = (Q * d) @ Q.T
    S = (S + S.T) / 2
    D, Y = eigh(H, S)
    check(S, D, Y, ref=d)


@pytest.mark.parametrize("n,b", [(16, 8), (40, 8), (48, 8), (64, 16)])
def test_small_diagonal_plus_border(H, n, b):
    """Step 15's shape: the previous Ritz values on the diagonal, k_b new columns."""
    rng = synth.rng(77 + n)
    S = np.diag(np.sort(rng.uniform(0, 2, n)))
    B = 1e-3 * rng.standard_normal((n, b))
    S[:, -b:] = B
    S[-b:, :] = B.T
    S[-b:, -b:] = (S[-b:, -b:] + S[-b:, -b:].T) / 2 + np.diag(rng.uniform(0, 2, b))
    D, Y = eigh(H, S)
    check(S, D, Y)


def test_small_repeated_calls_agree(H):
    """Same input, same output bits (the cluster's CTAs agree, no order-dependent sums)."""
    n = 48
    M = synth.rng(4).standard_normal((n, n))
    S = (M + M.T) / 2
    D1, Y1 = eigh(H, S)
    D2, Y2 = eigh(H, S)
    assert np.array_equal(D1, D2) and np.array_equal(Y1, Y2)
