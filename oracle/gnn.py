"""Learned start block for Algorithm 2: a message-passing network and its training loss.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper feeds Algorithm 2 an optional block of initial vectors V_init and filters them
progressively, best Rayleigh quotient first (Sec. 3, progressive filtering, Step 17).  This
module states, in plain float64 numpy, a small network that proposes such a block and the
quantities its training needs.  It is an extension of the method, not a step the paper
prints, so the definitions below are the specification both sides implement:

Inputs of graph G with Laplacian A (Eq. (1)), deg_i = number of neighbours of node i:
    X0 = [ sqrt(deg)/8 , log(1 + deg)/8 , R ]          (N x d_in, R: N x d_r random features)
Message passing on the normalised adjacency  Ahat = I - A  (L = 3 layers):
    S_l = (Ahat H_{l-1}) W_l + H_{l-1} U_l + 1 b_l^T ,   H_l = relu(S_l) ,   H_0 = X0
Output block:
    Z = H_L Wo                                           (N x k)
Loss against the solver's eigenvectors U (N x k, orthonormal columns):
    G = Z^T Z + rho I ,  rho = ridge * tr(Z^T Z) / k ,  P = U^T Z
    loss = 1 - tr(G^{-1} P^T P) / k
With rho = 0 this is 1 - (1/k) sum_i cos^2(theta_i), theta_i the principal angles between
span(Z) and span(U): 0 when span(Z) = span(U), 1 when they are orthogonal, independent of
the scale and of any invertible mixing of Z's columns.  Its gradient (rho held fixed):
    dloss/dZ = -(2/k) [ U P G^{-1} - Z G^{-1} P^T P G^{-1} ]
(the ridge term's own dependence on Z is excluded from the gradient on both sides).

Parameter order of the flat vector (float values, row-major matrices):
    W_1 (d_in x w), U_1 (d_in x w), b_1 (w), then for l = 2..L: W_l, U_l (w x w), b_l (w),
    then Wo (w x k).
"""
from __future__ import annotations

import numpy as np

N_LAYERS = 3


def param_shapes(d_in: int, width: int, k: int, layers: int = N_LAYERS):
    shapes = []
    p = d_in
    for _ in range(layers):
        shapes += [(p, width), (p, width), (width,)]
        p = width
    shapes.append((width, k))
    return shapes


def n_params(d_in: int, width: int, k: int, layers: int = N_LAYERS) -> int:
    return int(sum(int(np.prod(s)) for s in param_shapes(d_in, width, k, layers)))


def unpack(theta: np.ndarray, d_in: int, width: int, k: int, layers: int = N_LAYERS):
    """Flat parameter vector -> list of arrays in the documented order."""
    out, o = [], 0
    for s in param_shapes(d_in, width, k, layers):
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def features(L, R: np.ndarray) -> np.ndarray:
    """X0 = [sqrt(deg)/8, log(1+deg)/8, R]; deg from the Laplacian's off-diagonal pattern."""
    rowptr = L.rowptr
    deg = np.diff(rowptr).astype(np.float64)
    rows = np.repeat(np.arange(L.n), np.diff(rowptr))
    deg -= np.bincount(rows[L.colidx == rows], minlength=L.n)   # the stored diagonal
    return np.hstack([np.sqrt(deg)[:, None] / 8.0, np.log1p(deg)[:, None] / 8.0,
                      np.asarray(R, dtype=np.float64)])


def forward(A, X0: np.ndarray, theta: np.ndarray, width: int, k: int, layers: int = N_LAYERS):
    """Z and the per-layer cache (H_{l-1}, Ahat H_{l-1}, S_l) of the network above."""
    params = unpack(theta, X0.shape[1], width, k, layers)
    H = X0
    cache = []
    for l in range(layers):
        W, Uw, b = params[3 * l], params[3 * l + 1], params[3 * l + 2]
        AH = H - A @ H                     # Ahat H = (I - A) H
        S = AH @ W + H @ Uw + b[None, :]
        cache.append((H, AH, S))
        H = np.maximum(S, 0.0)
    Z = H @ params[-1]
    return Z, (cache, H, params)


def loss_and_dZ(Z: np.ndarray, U: np.ndarray, ridge: float = 1e-6):
    k = Z.shape[1]
    ZtZ = Z.T @ Z
    rho = ridge * np.trace(ZtZ) / k
    G = ZtZ + rho * np.eye(k)
    P = U.T @ Z
    Gi = np.linalg.inv(G)
    M = P.T @ P
    loss = 1.0 - np.trace(Gi @ M) / k
    dZ = -(2.0 / k) * (U @ (P @ Gi) - Z @ (Gi @ M @ Gi))
    return float(loss), dZ


def backward(A, dZ: np.ndarray, state, layers: int = N_LAYERS) -> np.ndarray:
    """Gradient of the loss with respect to the flat parameter vector, given dloss/dZ."""
    cache, HL, params = state
    grads = [None] * len(params)
    grads[-1] = HL.T @ dZ
    dH = dZ @ params[-1].T
    for l in reversed(range(layers)):
        H, AH, S = cache[l]
        W, Uw = params[3 * l], params[3 * l + 1]
        dS = dH * (S > 0.0)
        grads[3 * l] = AH.T @ dS
        grads[3 * l + 1] = H.T @ dS
        grads[3 * l + 2] = dS.sum(axis=0)
        if l > 0:
            T = dS @ W.T
            dH = (T - A @ T) + dS @ Uw.T   # Ahat^T = Ahat
    return np.concatenate([g.ravel() for g in grads])


def loss_and_grad(A, X0, theta, U, width, k, ridge=1e-6, layers: int = N_LAYERS):
    Z, state = forward(A, X0, theta, width, k, layers)
    loss, dZ = loss_and_dZ(Z, U, ridge)
    return loss, backward(A, dZ, state, layers), Z


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction; t counts from 1.
    Non-finite gradient components count as zero."""
    grad = np.where(np.isfinite(grad), grad, 0.0)
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def start_block(A, Z: np.ndarray):
    """Orthonormal basis of span(Z) rotated to its Ritz vectors, ascending Rayleigh quotients
    (the order the progressive filter expects of V_init)."""
    Q, _ = np.linalg.qr(Z)
    Hq = Q.T @ (A @ Q)
    w, Y = np.linalg.eigh(0.5 * (Hq + Hq.T))
    return Q @ Y, w
