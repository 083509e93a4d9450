"""Spectrum bounds by k-step Lanczos, for matrices whose bounds are not known analytically.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2: the filter's bounds a, a0 and b are analytic for the normalized Laplacian (0 and 2) and
otherwise estimated by standard Lanczos with a few matrix-vector products (the bound estimator
of the Chebyshev-Davidson work the paper cites; Zhou and Li, 2011).  Reading, shared with the
CUDA path:

Start vector v_1 = u / ||u|| with u entry i of Philox stream 3, vector 0, the solve's seed
(uniform in [-1/2, 1/2), oracle/philox.py).  For j = 1..k (plain three-term recurrence, no
reorthogonalisation; v_0 = 0, beta_0 = 0):
    w       = A v_j - beta_{j-1} v_{j-1}
    alpha_j = v_j . w
    w       = w - alpha_j v_j
    beta_j  = ||w||
    v_{j+1} = w / beta_j
An exactly zero beta_j ends the recurrence after step j (an invariant subspace).  With T_k the
symmetric tridiagonal matrix of alpha_1..alpha_k and beta_1..beta_{k-1}, and
theta_1 <= ... <= theta_k its eigenvalues:
    upperb = theta_k + beta_k      (theta_max + ||f_k||, f_k = beta_k v_{k+1} the residual of
                                    A V_k = V_k T_k + f_k e_k^T)
    lowb   = theta_1
and the first low_nwb = lowb + (upperb - lowb) k_want / N as for the analytic bounds.
"""
from __future__ import annotations

import numpy as np

from .philox import uniform_pm_half

STREAM_LANCZOS = 3


def start_vector(n: int, seed: int) -> np.ndarray:
    u = uniform_pm_half(n, 0, STREAM_LANCZOS, seed)
    return u / np.linalg.norm(u)


def lanczos(A, v1: np.ndarray, k: int):
    """(alpha, beta, V) of k steps (fewer when some beta_j is exactly 0); V is N x (steps + 1)."""
    n = v1.shape[0]
    V = [np.asarray(v1, dtype=np.float64)]
    alpha, beta = [], []
    v_prev = np.zeros(n)
    b_prev = 0.0
    for _ in range(k):
        v = V[-1]
        w = A @ v - b_prev * v_prev
        a = float(v @ w)
        w = w - a * v
        b = float(np.sqrt(w @ w))
        alpha.append(a)
        beta.append(b)
        if b == 0.0:
            V.append(np.zeros(n))
            break
        V.append(w / b)
        v_prev, b_prev = v, b
    return np.array(alpha), np.array(beta), np.stack(V, axis=1)


def tridiagonal(alpha: np.ndarray, beta: np.ndarray) -> np.ndarray:
    k = alpha.size
    return np.diag(alpha) + np.diag(beta[: k - 1], 1) + np.diag(beta[: k - 1], -1)


def bounds(A, k: int, seed: int):
    """(lowb, upperb, alpha, beta) of the k-step estimate from the seeded start vector."""
    n = A.shape[0]
    alpha, beta, _ = lanczos(A, start_vector(n, seed), k)
    theta = np.linalg.eigvalsh(tridiagonal(alpha, beta))
    return float(theta[0]), float(theta[-1] + beta[-1]), alpha, beta
