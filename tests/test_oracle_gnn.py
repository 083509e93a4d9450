"""Pins of the start-block network's oracle (oracle/gnn.py): central finite differences of
the loss through every parameter group, closed-form values of the subspace loss, and the
Ritz ordering of the start block."""
import numpy as np
import pytest

import oracle
import synth
from oracle import gnn


def _setup(n_graph=60, k=4, width=6, d_r=3, seed=0):
    g = synth.sbm_edges(n_graph, 3, d_in=5, d_out=1, seed=seed + 1)
    L = oracle.laplacian_csr(g.n, g.src, g.dst)
    A = L.scipy()
    X0 = gnn.features(L, synth.gnn_random_features(g.n, d_r, seed + 2))
    theta = synth.gnn_init(X0.shape[1], width, k, seed=seed + 3).astype(np.float64)
    w, Y = np.linalg.eigh(L.dense())
    U = Y[:, :k]
    return L, A, X0, theta, U, width, k


def test_features_closed_form():
    g = synth.star_edges(5)                           # hub degree 5, leaves degree 1
    L = oracle.laplacian_csr(g.n, g.src, g.dst)
    X0 = gnn.features(L, np.zeros((g.n, 2)))
    assert np.allclose(X0[0, :2], [np.sqrt(5) / 8, np.log(6) / 8])
    assert np.allclose(X0[1:, :2], [1 / 8, np.log(2) / 8])


def test_gradient_matches_central_differences():
    L, A, X0, theta, U, width, k = _setup()
    loss, grad, _ = gnn.loss_and_grad(A, X0, theta, U, width, k, ridge=0.0)
    rng = np.random.default_rng(5)
    offsets = np.cumsum([0] + [int(np.prod(s)) for s in gnn.param_shapes(X0.shape[1], width, k)])
    # a few coordinates of every parameter group (W, U, b of each layer, Wo)
    for gi in range(len(offsets) - 1):
        for idx in rng.integers(offsets[gi], offsets[gi + 1], 3):
            h = 1e-6
            tp, tm = theta.copy(), theta.copy()
            tp[idx] += h
            tm[idx] -= h
            fp = gnn.loss_and_dZ(gnn.forward(A, X0, tp, width, k)[0], U, 0.0)[0]
            fm = gnn.loss_and_dZ(gnn.forward(A, X0, tm, width, k)[0], U, 0.0)[0]
            fd = (fp - fm) / (2 * h)
            assert abs(fd - grad[idx]) <= 1e-6 * max(1.0, abs(fd)), (gi, idx, fd, grad[idx])


def test_loss_closed_forms():
    rng = np.random.default_rng(1)
    n, k = 50, 5
    Q, _ = np.linalg.qr(rng.standard_normal((n, 2 * k)))
    U, Uperp = Q[:, :k], Q[:, k:]
    C = rng.standard_normal((k, k)) + 3 * np.eye(k)
    assert abs(gnn.loss_and_dZ(U @ C, U, 0.0)[0]) < 1e-12          # same span
    assert abs(gnn.loss_and_dZ(7.5 * Uperp @ C, U, 0.0)[0] - 1.0) < 1e-12   # orthogonal span
    # one principal angle theta in each of the k planes: loss = mean sin^2(theta)
    th = np.linspace(0.1, 1.2, k)
    Z = U * np.cos(th) + Uperp * np.sin(th)
    assert abs(gnn.loss_and_dZ(Z, U, 0.0)[0] - np.mean(np.sin(th) ** 2)) < 1e-12
    # the gradient vanishes at the optimum and is orthogonal to Z (scale invariance)
    _, dZ = gnn.loss_and_dZ(U @ C, U, 0.0)
    assert np.abs(dZ).max() < 1e-9                    # rounding of G^{-1} (cond(C) ~ 10)
    _, dZ = gnn.loss_and_dZ(Z, U, 0.0)
    assert abs(np.sum(dZ * Z)) < 1e-12


def test_dZ_matches_central_differences_with_ridge():
    rng = np.random.default_rng(2)
    n, k = 40, 3
    U, _ = np.linalg.qr(rng.standard_normal((n, k)))
    Z = rng.standard_normal((n, k))
    _, dZ = gnn.loss_and_dZ(Z, U, 0.0)
    for (i, j) in [(0, 0), (7, 2), (39, 1)]:
        h = 1e-6
        Zp, Zm = Z.copy(), Z.copy()
        Zp[i, j] += h
        Zm[i, j] -= h
        fd = (gnn.loss_and_dZ(Zp, U, 0.0)[0] - gnn.loss_and_dZ(Zm, U, 0.0)[0]) / (2 * h)
        assert abs(fd - dZ[i, j]) < 1e-7


def test_adam_first_step_is_lr_times_sign():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    new, m, v = gnn.adam_step(theta, g, np.zeros(3), np.zeros(3), 1, 0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2, update = lr * g / (|g| + eps)
    assert np.allclose(new, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_start_block_is_ritz_ordered():
    L, A, X0, theta, U, width, k = _setup(k=5)
    Z = gnn.forward(A, X0, theta, width, k)[0]
    V, w = gnn.start_block(A, Z)
    assert np.all(np.diff(w) >= 0)
    assert np.abs(V.T @ V - np.eye(k)).max() < 1e-12
    assert np.allclose(np.diag(V.T @ (A @ V)), w)
    # span unchanged
    P = V @ (V.T @ Z)
    assert np.abs(P - Z).max() < 1e-10 * np.abs(Z).max()
