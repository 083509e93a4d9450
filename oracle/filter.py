"""Chebyshev polynomial filter: Algorithm 3 and the closed form it applies.

Reading of the arguments (the call in Algorithm 2, Step 5 lists them in a
different order from Algorithm 3's signature): the damped interval is
[a, b] = [low_nwb, upperb], a0 = lowb is the lower end of the whole spectrum,
so c = (a + b)/2, e = (b - a)/2 map [a, b] onto [-1, 1] and the wanted end
[a0, a) lands outside it where the Chebyshev polynomial grows.  The symbol
tau of the loop is the scalar t = 2/sigma fixed before the loop, and the
lower-case v of the update is the previous iterate.
"""
from __future__ import annotations

import numpy as np


def chebyshev_filter(A, X: np.ndarray, m: int, a: float, b: float, a0: float) -> np.ndarray:
    """Algorithm 3: returns p_m(A) X with p_m(x) = T_m((x-c)/e) / T_m((a0-c)/e).

    ``A`` is anything supporting ``A @ block`` (a scipy CSR matrix here).
    """
    if m < 1:
        raise ValueError("degree m must be >= 1")
    c = (a + b) / 2.0
    e = (b - a) / 2.0
    sigma = e / (a0 - c)
    tau = 2.0 / sigma
    V = np.array(X, dtype=np.float64, copy=True)
    U = (A @ V - c * V) * (sigma / e)
    for _ in range(2, m + 1):
        sigma1 = 1.0 / (tau - sigma)
        W = (A @ U - c * U) * (2.0 * sigma1 / e) - (sigma * sigma1) * V
        V = U
        U = W
        sigma = sigma1
    return U


def chebyshev_T(m: int, x):
    """Eq. (4): C_m(x) = cos(m arccos x) on [-1, 1], cosh(m arccosh |x|) (signed) outside."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(m * np.arccos(x[inside]))
    xo = x[~inside]
    sgn = np.where(xo < 0, (-1.0) ** m, 1.0)
    out[~inside] = sgn * np.cosh(m * np.arccosh(np.abs(xo)))
    return out


def filter_polynomial(lam, m: int, a: float, b: float, a0: float):
    """Closed form of the filter as a scalar polynomial (Eqs. (3)-(4))."""
    c = (a + b) / 2.0
    e = (b - a) / 2.0
    lam = np.asarray(lam, dtype=np.float64)
    return chebyshev_T(m, (lam - c) / e) / chebyshev_T(m, np.array([(a0 - c) / e]))[0]
