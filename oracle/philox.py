"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy
as 1, 2, 3", SC 2011), written from its published definition.

Used by the method for the random vectors it draws itself (replacement of
numerically dependent vectors in the orthonormalisation, Sec. 2, and the
columns Step 2 of Algorithm 2 constructs when fewer than k_b initial vectors
are given).  Entry (row i, vector number r) of a random vector of stream s and
seed q is

    (x0, x1, x2, x3) = Philox4x32-10(counter = (i, r, s, 0), key = (q mod 2^32, q >> 32))
    u = ((x0 >> 5) * 2^26 + (x1 >> 6)) * 2^-53 - 1/2,

an exactly representable value in [-1/2, 1/2).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)

STREAM_REPLACE = 1
STREAM_FILL = 2


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32 with 10 rounds; all arguments uint32-valued arrays/scalars."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK
    c1 = np.asarray(c1, dtype=np.uint64) & MASK
    c2 = np.asarray(c2, dtype=np.uint64) & MASK
    c3 = np.asarray(c3, dtype=np.uint64) & MASK
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0          # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def uniform_pm_half(n_rows: int, vec_index: int, stream: int, seed: int) -> np.ndarray:
    """Random vector number ``vec_index`` of ``stream``: n_rows values in [-1/2, 1/2)."""
    i = np.arange(n_rows, dtype=np.uint64)
    q = int(seed) & 0xFFFFFFFFFFFFFFFF
    x0, x1, _, _ = philox4x32_10(i, np.uint64(vec_index), np.uint64(stream), np.uint64(0),
                                 q & 0xFFFFFFFF, q >> 32)
    u53 = ((x0 >> np.uint64(5)) << np.uint64(26)) | (x1 >> np.uint64(6))
    return u53.astype(np.float64) * (2.0 ** -53) - 0.5
