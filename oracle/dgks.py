"""Orthonormalisation of a new block against the basis (Algorithm 2, Step 6).

The paper performs this step with DGKS (Daniel, Gragg, Kaufman, Stewart 1976)
and replaces vectors that have become numerically dependent on the basis by
random vectors (Sec. 2, "Orthonormalization").  Restated column by column:

    for each new column x (in order):
        project x against the current basis Q = [V, columns accepted so far]
        (classical Gram-Schmidt); if the norm fell below eta * (norm before),
        project once more (the DGKS criterion, eta = 1/sqrt(2));
        if what is left is below tau_dep * (original norm), or the original
        norm is zero, x is numerically dependent: replace it by the next
        random vector and start over with that vector;
        normalise and append to Q.

In exact arithmetic this yields the unique Gram-Schmidt basis of
[V, X] (with replacements), whatever blocking an implementation uses.
"""
from __future__ import annotations

import math

import numpy as np

from .philox import uniform_pm_half, STREAM_REPLACE

ETA = 1.0 / math.sqrt(2.0)
TAU_DEP_F64 = 1e-10


def dgks_orthonormalize(V: np.ndarray, X: np.ndarray, *, seed: int = 0, rep_counter: int = 0,
                        tau_dep: float = TAU_DEP_F64, max_replace: int = 8):
    """Return (Q, n_replaced, rep_counter): Q orthonormal, orthogonal to V's columns.

    V: N x k with orthonormal columns (k may be 0).  X: N x b.
    """
    N, b = X.shape
    cols = []
    basis = np.array(V, dtype=np.float64, copy=True).reshape(N, -1)
    n_rep = 0
    for j in range(b):
        x = np.array(X[:, j], dtype=np.float64, copy=True)
        for _attempt in range(max_replace + 1):
            nrm0 = float(np.linalg.norm(x))
            nrm = nrm0
            if basis.shape[1] > 0 and nrm0 > 0.0:
                x = x - basis @ (basis.T @ x)
                nrm = float(np.linalg.norm(x))
                if nrm < ETA * nrm0:
                    x = x - basis @ (basis.T @ x)
                    nrm = float(np.linalg.norm(x))
            if nrm0 > 0.0 and nrm > tau_dep * nrm0:
                break
            x = uniform_pm_half(N, rep_counter, STREAM_REPLACE, seed)
            rep_counter += 1
            n_rep += 1
        else:
            raise RuntimeError("orthonormalisation: replacement vectors keep failing")
        q = x / nrm
        cols.append(q)
        basis = np.concatenate([basis, q[:, None]], axis=1)
    Q = np.stack(cols, axis=1) if cols else np.zeros((N, 0))
    return Q, n_rep, rep_counter
