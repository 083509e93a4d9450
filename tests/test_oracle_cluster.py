"""Pins of the spectral-clustering oracle (oracle/cluster.py, Algorithm 1 Steps 4-5): scalar
brute force of the float32 distance and of the seeding, hand-computed k-means runs and scores,
library scores, invariants of Lloyd's iteration and planted-partition recovery."""
import numpy as np
import pytest

import oracle
import synth
from oracle import cluster as C


def test_normalize_rows_closed_form():
    V = np.array([[3.0, 4.0], [0.0, 0.0], [-2.0, 0.0], [1e-200, 1e-200], [0.0, 4.0],
                  [1.0, 1.0]])
    X = C.normalize_rows(V)
    assert np.allclose(X[0], [0.6, 0.8], rtol=2.3e-16, atol=0)   # 1/5 is not exact: 1 ulp
    assert np.array_equal(X[1], [0.0, 0.0])          # zero row stays zero
    assert np.array_equal(X[2], [-1.0, 0.0])
    assert np.array_equal(X[3], [0.0, 0.0])          # squares underflow: norm 0, row zero
    assert np.array_equal(X[4], [0.0, 1.0])          # r = 1/4 exact
    # 1/sqrt(2) rounded once, then the product: the float64 nearest 2^-1/2 here
    assert X[5, 0] == X[5, 1] == 1.0 / np.sqrt(2.0)
    assert C.features(V)[0].tolist() == [np.float32(0.6), np.float32(0.8)]


def test_normalize_rows_unit_length_and_direction():
    V = synth.gaussian_block(500, 7, seed=3)
    X = C.normalize_rows(V)
    nrm = np.linalg.norm(V, axis=1)
    assert np.allclose(np.linalg.norm(X, axis=1), 1.0, atol=1e-15, rtol=0)
    assert np.allclose(X * nrm[:, None], V, rtol=1e-15, atol=0)
    assert C.features(V).dtype == np.float32


def _scalar_dist(x, c):
    acc = np.float32(0.0)
    for xd, cd in zip(x, c):
        diff = np.float32(np.float32(xd) - np.float32(cd))
        acc = np.float32(acc + np.float32(diff * diff))
    return acc


def test_distance_matches_scalar_float32_loop():
    X = synth.gaussian_block(40, 9, seed=4).astype(np.float32)
    c = X[7]
    got = C.dist_to(X, c)
    want = np.array([_scalar_dist(X[i], c) for i in range(40)], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    exact = np.sum((X.astype(np.float64) - c.astype(np.float64)) ** 2, axis=1)
    assert np.allclose(got, exact, rtol=1e-5, atol=0)


def test_assign_brute_force_and_ties():
    X = synth.gaussian_block(60, 5, seed=5).astype(np.float32)
    Cen = np.vstack([X[3], X[10], X[10], X[40]]).astype(np.float64)   # rows 1 and 2 tie
    lab = C.assign(X, Cen)
    for i in range(60):
        d = [_scalar_dist(X[i], Cen[j].astype(np.float32)) for j in range(4)]
        assert lab[i] == int(np.argmin(d))            # argmin: first minimum
    assert not np.any(lab == 2)                       # duplicate centroid never wins a tie
    assert lab[10] == 1 and lab[3] == 0 and lab[40] == 3


def test_farthest_first_closed_form():
    X = (np.array([[0.0], [1.0], [2.0], [10.0], [2.0]]) / 16).astype(np.float32)
    # from 0: farthest is 10 (index 3); then min distances 1, 4, 0, 4 -> first of the
    # tied 2's (index 2); then 1 is the only point left at distance 1
    assert C.farthest_first(X, 0, 4).tolist() == [0, 3, 2, 1]


def test_farthest_first_brute_force():
    X = synth.gaussian_block(30, 3, seed=6).astype(np.float32)
    got = C.farthest_first(X, 11, 6)
    seeds = [11]
    for _ in range(5):
        best, arg = -1.0, -1
        for i in range(30):
            m = min(_scalar_dist(X[i], X[s]) for s in seeds)
            if m > best:
                best, arg = m, i
        seeds.append(arg)
    assert got.tolist() == seeds


def test_kmeans_hand_example():
    pts = np.array([1, 2, 3, 10, 11, 12], dtype=np.float64) / 16
    X = pts[:, None].astype(np.float32)
    # round 1 from seeds {1, 2}: labels 0,1,1,1,1,1; centroids 1 and 7.6; round 2: 0,0,0,1,1,1;
    # centroids 2 and 11; round 3 changes nothing
    lab, Cen, rounds = C.kmeans(X, np.array([0, 1]), 100)
    assert lab.tolist() == [0, 0, 0, 1, 1, 1]
    assert rounds == 3
    assert np.array_equal(Cen[:, 0], [2 / 16, 11 / 16])
    lab1, _, r1 = C.kmeans(X, np.array([0, 1]), 1)
    assert r1 == 1 and lab1.tolist() == [0, 1, 1, 1, 1, 1]


def test_update_is_the_mean_and_keeps_empty_clusters():
    X = synth.gaussian_block(2000, 6, seed=7)
    X = (X / np.abs(X).max()).astype(np.float32)
    lab = synth.rng(8).integers(0, 5, 2000).astype(np.int32)
    lab[lab == 3] = 4                                 # cluster 3 empty
    prev = np.full((6, 6), 0.25)
    newC = C.update(X, lab, prev)
    for j in (0, 1, 2, 4):
        mean = X[lab == j].astype(np.float64).mean(axis=0)
        assert np.max(np.abs(newC[j] - mean)) <= 2.0 ** -37 * (1 + 1e-9)
    assert np.array_equal(newC[3], prev[3]) and np.array_equal(newC[5], prev[5])
    perm = synth.rng(9).permutation(2000)            # integer sums: order-independent bits
    assert np.array_equal(C.update(X[perm], lab[perm], prev), newC)


def test_lloyd_invariants():
    X = C.features(synth.gaussian_block(3000, 4, seed=10))
    seeds = C.farthest_first(X, 5, 6)
    prev = np.inf
    for r in range(1, 8):
        lab, Cen, rounds = C.kmeans(X, seeds, r)
        # objective of the labels with their own means never rises (Lloyd's descent)
        obj = C.objective(X, lab, C.update(X, lab, Cen))
        assert obj <= prev * (1 + 1e-6)
        prev = obj
    lab, Cen, rounds = C.kmeans(X, seeds, 200)
    assert rounds < 200
    assert np.array_equal(C.assign(X, Cen), lab)                 # fixed point
    assert np.array_equal(C.update(X, lab, Cen), Cen)


def test_kmeans_recovers_separated_blobs():
    g = synth.rng(11)
    centers = np.eye(8) * 0.9
    truth = g.integers(0, 8, 4000)
    X = (centers[truth] + 0.02 * g.standard_normal((4000, 8))).astype(np.float32)
    lab, _, _ = C.kmeans(X, C.farthest_first(X, 0, 8), 100)
    assert C.adjusted_rand_index(lab, truth) == 1.0
    assert C.normalized_mutual_info(lab, truth) == pytest.approx(1.0, abs=1e-12)


def test_scores_hand_computed():
    a, b = [0, 0, 1, 1], [0, 0, 1, 2]
    assert C.adjusted_rand_index(a, b) == pytest.approx(4 / 7, abs=1e-15)
    assert C.normalized_mutual_info(a, b) == pytest.approx(0.8, abs=1e-15)
    assert C.adjusted_rand_index([0, 0, 1, 1], [0, 1, 0, 1]) == pytest.approx(-0.5, abs=1e-15)
    assert C.normalized_mutual_info([0, 0, 1, 1], [0, 1, 0, 1]) == pytest.approx(0.0, abs=1e-15)
    assert C.adjusted_rand_index([0, 0, 1, 2], [5, 5, 7, 3]) == 1.0   # relabelling
    assert C.normalized_mutual_info([0, 0, 1, 2], [5, 5, 7, 3]) == pytest.approx(1.0)


def test_scores_match_scikit_learn():
    metrics = pytest.importorskip("sklearn.metrics")
    g = synth.rng(12)
    for t in range(5):
        a = g.integers(0, 6, 500)
        b = np.where(g.random(500) < 0.6, a, g.integers(0, 9, 500))
        assert C.adjusted_rand_index(a, b) == pytest.approx(metrics.adjusted_rand_score(a, b),
                                                             abs=1e-12)
        assert C.normalized_mutual_info(a, b) == pytest.approx(
            metrics.normalized_mutual_info_score(a, b), abs=1e-12)


def test_spectral_clustering_recovers_planted_partition():
    g = synth.sbm_edges(600, 4, d_in=20.0, d_out=1.0, seed=13)
    L = oracle.laplacian_csr(g.n, g.src, g.dst)
    w, Y = np.linalg.eigh(L.dense())
    lab, _, rounds, seeds = C.spectral_cluster(Y[:, :4], 4, 17)
    assert sorted(g.labels[seeds].tolist()) == [0, 1, 2, 3]
    assert C.adjusted_rand_index(lab, g.labels) == 1.0
    assert rounds <= 3
