"""Pins of the oracle's orthonormalisation (Algorithm 2, Step 6) and of its Philox generator."""
import numpy as np
import pytest

import synth
from oracle import dgks_orthonormalize, philox4x32_10, uniform_pm_half


def test_philox_known_answers():
    # Known-answer vectors published with the Random123 library for Philox4x32-10.
    cases = [
        ((0, 0, 0, 0, 0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 6, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344, 0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for args, expect in cases:
        got = tuple(int(x) for x in philox4x32_10(*args))
        assert got == expect


def test_uniform_range_and_moments():
    u = uniform_pm_half(200000, 3, 1, 99)
    assert u.min() >= -0.5 and u.max() < 0.5
    assert abs(u.mean()) < 5e-3 and abs(u.var() - 1 / 12) < 2e-3
    assert not np.array_equal(u, uniform_pm_half(200000, 4, 1, 99))


def _orth_basis(n, k, seed):
    Q, _ = np.linalg.qr(synth.gaussian_block(n, k, seed))
    return Q


@pytest.mark.parametrize("k,b", [(0, 5), (12, 4), (40, 10)])
def test_orthonormal_and_span(k, b):
    n = 300
    V = _orth_basis(n, k, 1)
    X = synth.gaussian_block(n, b, 2)
    Q, nrep, _ = dgks_orthonormalize(V, X)
    assert nrep == 0
    assert np.abs(Q.T @ Q - np.eye(b)).max() < 1e-14
    if k:
        assert np.abs(V.T @ Q).max() < 1e-14
    B = np.concatenate([V, Q], 1)
    assert np.abs(X - B @ (B.T @ X)).max() < 1e-12 * np.abs(X).max()


def test_matches_householder_qr_without_basis():
    X = synth.gaussian_block(200, 6, 5)
    Q, _, _ = dgks_orthonormalize(np.zeros((200, 0)), X)
    Qh, R = np.linalg.qr(X)
    Qh = Qh * np.sign(np.diag(R))[None, :]
    assert np.abs(Q - Qh).max() < 1e-13


def test_orthogonal_input_passes_unchanged():
    n = 120
    B = _orth_basis(n, 10, 3)
    V, X = B[:, :6], B[:, 6:]
    Q, nrep, _ = dgks_orthonormalize(V, X)
    assert nrep == 0 and np.abs(Q - X).max() < 1e-14


def test_dependent_columns_replaced():
    n = 150
    V = _orth_basis(n, 8, 4)
    X = synth.gaussian_block(n, 4, 6)
    X[:, 1] = X[:, 0] * 3.0           # duplicate of an earlier new column
    X[:, 2] = V[:, 5] + 1e-14 * X[:, 3]   # (numerically) inside span(V)
    X[:, 3] = 0.0                     # zero column
    Q, nrep, ctr = dgks_orthonormalize(V, X, seed=7, rep_counter=10)
    assert nrep == 3 and ctr == 13
    assert np.abs(Q.T @ Q - np.eye(4)).max() < 1e-14
    assert np.abs(V.T @ Q).max() < 1e-14
