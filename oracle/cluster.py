"""Spectral clustering after the eigensolver: Algorithm 1, Steps 4 and 5.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Step 4 scales each row of the N x k eigenvector block to unit Euclidean length; the rows are
the nodes' features.  Step 5 clusters the features, with k-means named as one choice.  The paper
fixes neither the k-means variant, its seeding nor its arithmetic, so this module is the
definition that the CUDA path reproduces bit for bit:

Features (Step 4).  s_i = sum over d = 0..k-1, in that order, of V_id * V_id in float64 (each
product and sum rounded, no fused multiply-add); r_i = 1 / sqrt(s_i) (one float64 square root
and one division per row); X_id = float32(V_id * r_i) (float64 product, then round to nearest
float32); a row with s_i = 0 stays zero.

Distance.  dist(x, c) in float32: acc = 0; for d = 0..k-1: diff = x_d - c_d;
acc = acc + diff * diff, every operation rounded to float32, no fused multiply-add.

Seeding (farthest-first traversal, Gonzalez 1985).  s_0 = ``first`` (a seeded draw of the
caller); dmin_i = +inf; for j = 1..c-1: dmin_i = min(dmin_i, dist(X_i, X_{s_{j-1}})) and
s_j = argmax_i dmin_i, the lowest i on ties.

Lloyd's iteration.  Centroids start at C_j = X_{s_j} (float64).  Assignment: label_i = argmin_j
dist(X_i, float32(C_j)), the lowest j on ties.  Update: q_id = round-half-even(X_id * 2^36) as a
64-bit integer, Q_jd = sum of q_id over the members of cluster j (an integer sum, the same in
any order; it cannot overflow while |X_id| <= 1, as for Step 4's rows, and N < 2^27),
C_jd = (float64(Q_jd) / count_j) * 2^-36; a cluster without members keeps its centroid.  The
fixed-point mean differs from the float64 mean by at most 2^-37 per coordinate, far below the
float32 resolution of the assignment; it makes the centroids independent of the summation
order.  Rounds: the first assignment is round 1; each update followed by an assignment is one
more round; stop when an assignment changes no label or after ``max_rounds`` rounds.

Also the two scores used against planted labels: the adjusted Rand index (Hubert and Arabie,
1985) and normalised mutual information with the arithmetic-mean normalisation.
"""
from __future__ import annotations

import numpy as np

Q_SCALE = 2.0 ** 36


def normalize_rows(V: np.ndarray) -> np.ndarray:
    """Step 4 in float64: rows of V scaled to unit length (sequential sum of squares)."""
    V = np.asarray(V, dtype=np.float64)
    s = np.zeros(V.shape[0])
    for d in range(V.shape[1]):
        s = s + V[:, d] * V[:, d]
    out = np.zeros_like(V)
    nz = s > 0
    r = 1.0 / np.sqrt(s[nz])
    out[nz] = V[nz] * r[:, None]
    return out


def features(V: np.ndarray) -> np.ndarray:
    """float32 features X of Step 4 (N x k)."""
    return normalize_rows(V).astype(np.float32)


def dist_to(X: np.ndarray, c: np.ndarray) -> np.ndarray:
    """float32 squared distances of every row of X to the point c, in the order defined above."""
    X = np.asarray(X, dtype=np.float32)
    c = np.asarray(c, dtype=np.float32)
    acc = np.zeros(X.shape[0], dtype=np.float32)
    for d in range(X.shape[1]):
        diff = X[:, d] - c[d]
        acc = acc + diff * diff
    return acc


def farthest_first(X: np.ndarray, first: int, n_clusters: int) -> np.ndarray:
    X = np.asarray(X, dtype=np.float32)
    seeds = [int(first)]
    dmin = np.full(X.shape[0], np.inf, dtype=np.float32)
    for _ in range(1, n_clusters):
        dmin = np.minimum(dmin, dist_to(X, X[seeds[-1]]))
        seeds.append(int(np.argmax(dmin)))      # first maximum: lowest index on ties
    return np.asarray(seeds, dtype=np.int32)


def assign(X: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Nearest centroid of every row (float32 distance; ties to the lowest centroid index)."""
    C32 = np.asarray(C, dtype=np.float64).astype(np.float32)
    best = np.full(X.shape[0], np.inf, dtype=np.float32)
    lab = np.zeros(X.shape[0], dtype=np.int32)
    for j in range(C32.shape[0]):
        acc = dist_to(X, C32[j])
        better = acc < best
        best = np.where(better, acc, best)
        lab = np.where(better, np.int32(j), lab)
    return lab


def quantize(X: np.ndarray) -> np.ndarray:
    return np.rint(np.asarray(X, dtype=np.float32).astype(np.float64) * Q_SCALE).astype(np.int64)


def update(X: np.ndarray, lab: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Centroids as the fixed-point means of their members; empty clusters keep theirs."""
    q = quantize(X)
    newC = np.array(C, dtype=np.float64, copy=True)
    for j in range(newC.shape[0]):
        m = lab == j
        cnt = int(np.count_nonzero(m))
        if cnt:
            Q = q[m].sum(axis=0, dtype=np.int64)
            newC[j] = (Q.astype(np.float64) / float(cnt)) * (1.0 / Q_SCALE)
    return newC


def kmeans(X: np.ndarray, seeds: np.ndarray, max_rounds: int = 100):
    """Lloyd's k-means from the rows ``seeds`` of X; returns (labels, centroids, rounds) with
    the centroids of the last assignment."""
    X = np.asarray(X, dtype=np.float32)
    C = X[np.asarray(seeds)].astype(np.float64)
    lab = assign(X, C)
    rounds = 1
    while rounds < max_rounds:
        C = update(X, lab, C)
        new = assign(X, C)
        rounds += 1
        same = np.array_equal(new, lab)
        lab = new
        if same:
            break
    return lab, C, rounds


def spectral_cluster(V: np.ndarray, n_clusters: int, first: int, max_rounds: int = 100):
    """Steps 4 and 5: features, farthest-first seeds, Lloyd's k-means."""
    X = features(V)
    seeds = farthest_first(X, first, n_clusters)
    lab, C, rounds = kmeans(X, seeds, max_rounds)
    return lab, C, rounds, seeds


def objective(X: np.ndarray, lab: np.ndarray, C: np.ndarray) -> float:
    """Sum of squared float64 distances of the rows to their centroids."""
    X = np.asarray(X, dtype=np.float64)
    return float(np.sum((X - np.asarray(C, dtype=np.float64)[lab]) ** 2))


def _contingency(a, b):
    _, ia = np.unique(np.asarray(a), return_inverse=True)
    _, ib = np.unique(np.asarray(b), return_inverse=True)
    M = np.zeros((ia.max() + 1, ib.max() + 1), dtype=np.int64)
    np.add.at(M, (ia, ib), 1)
    return M


def adjusted_rand_index(a, b) -> float:
    """(I - E) / (mean(A, B) - E) over pair counts (Hubert and Arabie, 1985)."""
    M = _contingency(a, b).astype(np.float64)
    pairs = lambda x: x * (x - 1.0) / 2.0
    I = pairs(M).sum()
    A = pairs(M.sum(axis=1)).sum()
    B = pairs(M.sum(axis=0)).sum()
    E = A * B / pairs(M.sum())
    if 0.5 * (A + B) == E:
        return 1.0
    return float((I - E) / (0.5 * (A + B) - E))


def normalized_mutual_info(a, b) -> float:
    """2 I(a; b) / (H(a) + H(b)) with natural logarithms."""
    P = _contingency(a, b).astype(np.float64)
    P /= P.sum()
    pa, pb = P.sum(axis=1), P.sum(axis=0)
    nz = P > 0
    mi = float(np.sum(P[nz] * np.log(P[nz] / np.outer(pa, pb)[nz])))
    ha = -float(np.sum(pa * np.log(pa)))
    hb = -float(np.sum(pb * np.log(pb)))
    if ha + hb == 0.0:
        return 1.0
    return 2.0 * mi / (ha + hb)
