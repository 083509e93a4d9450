"""Spectral clustering on the GPU (bchdav_row_normalize, bchdav_kmeans_seed, bchdav_kmeans,
bchdav_spectral_cluster; Algorithm 1, Steps 4-5) against the oracle (oracle/cluster.py):
bit-exact features, seeds, labels, centroids and round counts on seeded inputs; properties at
the size of the 1M-node, 100-cluster workload; planted-partition recovery after the GPU
eigensolver."""
import numpy as np
import pytest

import synth
from gpu_util import device_csr, to_np
from oracle import cluster as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import paper_2212_04443_gb300 as P
    return P.Handle()


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32 if a.dtype == np.float32 else np.uint64)


@pytest.mark.parametrize("n,dim,ldpad", [(1, 1, 0), (5003, 7, 3), (20011, 100, 0),
                                         (777, 130, 1), (300, 512, 0)])
def test_row_normalize_bit_exact(H, n, dim, ldpad):
    import torch
    V = synth.gaussian_block(n, dim, seed=n + dim)
    g = synth.rng(n)
    V[g.integers(0, n, 3)] = 0.0                    # zero rows stay zero
    V[g.integers(0, n, 2)] = 1e-200                 # squares underflow: zero rows too
    V[g.integers(0, n, 2)] *= 1e150
    Vd = torch.zeros((n, dim + ldpad), dtype=torch.float64, device="cuda")
    Vd[:, :dim] = _cuda(V)
    Xt = H.row_normalize(Vd[:, :dim])
    assert np.array_equal(_bits(to_np(Xt).T), _bits(C.features(V)))


def _tied_features(n, dim, seed):
    """Coarse values: many exactly equal distances, so every tie rule is exercised."""
    X = np.round(synth.gaussian_block(n, dim, seed) * 2) / 8
    return np.clip(X, -1, 1).astype(np.float32)


@pytest.mark.parametrize("case", ["planted", "planted_n4", "ties", "ties_n4", "single"])
def test_seeds_bit_exact(H, case):
    # n % 4 == 0 takes the four-nodes-per-thread pass, other n the one-node pass
    if case.startswith("planted"):
        n = 30012 if case.endswith("n4") else 30011
        V, _ = synth.planted_embedding(n, 20, 20, noise=0.3, seed=3, contiguous=False)
        X, c, first = C.features(V), 20, 12345
    elif case == "ties_n4":
        X, c, first = _tied_features(4100, 3, 4), 12, 7
    elif case == "ties":
        X, c, first = _tied_features(4099, 3, 4), 12, 7
    else:
        X, c, first = _tied_features(50, 2, 5), 1, 49
    seeds = H.kmeans_seed(_cuda(X.T), c, first)
    assert to_np(seeds).tolist() == C.farthest_first(X, first, c).tolist()


KM_CASES = [
    # n, dim, clusters, contiguous labels, max rounds, noise (None: unclustered Gaussian rows)
    (30011, 20, 20, True, 100, 1.2),      # 14 rounds; warps share labels; sums in shared memory
    (30011, 20, 20, False, 100, 1.2),     # mixed warps: one atomic per node
    (20011, 100, 100, True, 100, 1.6),    # 15 rounds; sums over 48 KB: global atomics
    (20011, 100, 100, False, 100, 1.2),
    (4099, 3, 37, False, 200, None),      # about 50 rounds; 37 clusters pad the block of 20
    (4099, 3, 37, False, 3, None),        # stopped by max_rounds
    (2500, 130, 7, True, 100, 1.0),       # dim > 128
    (1000, 5, 1, True, 100, None),        # one cluster
    (5000, 200, 200, False, 4, 2.5),      # centroids over 96 KB: blocks staged in turn
    (3000, 512, 10, True, 100, 1.0),      # the largest dimension
]


@pytest.mark.parametrize("n,dim,c,contig,rounds,noise", KM_CASES)
def test_kmeans_bit_exact(H, n, dim, c, contig, rounds, noise):
    if noise is None:
        X = C.features(synth.gaussian_block(n, dim, seed=n))
    else:
        V, _ = synth.planted_embedding(n, c, dim, noise=noise, seed=n + c, contiguous=contig)
        X = C.features(V)
    seeds = C.farthest_first(X, n // 3, c)
    lab, cent, r = H.kmeans(_cuda(X.T), _cuda(seeds), rounds)
    lab_o, cent_o, r_o = C.kmeans(X, seeds, rounds)
    assert r == r_o
    assert np.array_equal(to_np(lab), lab_o)
    assert np.array_equal(_bits(to_np(cent)), _bits(cent_o))


def test_kmeans_empty_cluster_keeps_its_centroid(H):
    X = _tied_features(3001, 4, 6)
    seeds = np.array([5, 100, 5, 2000], dtype=np.int32)   # cluster 2 duplicates cluster 0
    # round 1 leaves cluster 2 empty (ties go to cluster 0), so the centroids of round 2 keep
    # its seed; later rounds give it members once cluster 0 has moved
    for rounds in (2, 50):
        lab, cent, r = H.kmeans(_cuda(X.T), _cuda(seeds), rounds)
        lab_o, cent_o, r_o = C.kmeans(X, seeds, rounds)
        assert r == r_o and np.array_equal(to_np(lab), lab_o)
        assert np.array_equal(_bits(to_np(cent)), _bits(cent_o))
        if rounds == 2:
            assert np.array_equal(cent_o[2], X[5].astype(np.float64))
            assert not np.array_equal(cent_o[0], X[5].astype(np.float64))


def test_kmeans_seed_out_of_range_is_an_error(H):
    X = _tied_features(1000, 3, 7)
    import paper_2212_04443_gb300 as P
    with pytest.raises(P.BchdavError, match="seed"):
        H.kmeans(_cuda(X.T), _cuda(np.array([0, 1000], dtype=np.int32)), 5)
    # the handle stays usable
    lab, _, _ = H.kmeans(_cuda(X.T), _cuda(np.array([0, 999], dtype=np.int32)), 5)
    assert np.array_equal(to_np(lab), C.kmeans(X, np.array([0, 999]), 5)[0])


def test_spectral_cluster_one_call_matches_oracle(H):
    V, truth = synth.planted_embedding(50021, 50, 50, noise=0.5, seed=8, contiguous=False)
    lab, cent, seeds, r = H.spectral_cluster(_cuda(V), 50, 999)
    lab_o, cent_o, r_o, seeds_o = C.spectral_cluster(V, 50, 999)
    assert to_np(seeds).tolist() == seeds_o.tolist()
    assert r == r_o and np.array_equal(to_np(lab), lab_o)
    assert np.array_equal(_bits(to_np(cent)), _bits(cent_o))
    assert C.adjusted_rand_index(lab_o, truth) == 1.0


def test_full_size_properties(H):
    """1M nodes, 100 clusters, 100 dimensions (the shape of the 1M-node SBM's eigenvectors):
    sampled features bit-exact, sampled labels nearest to the returned centroids, every
    centroid the mean of its members, planted partition recovered."""
    n, c = 1_000_000, 100
    V, truth = synth.planted_embedding(n, c, c, noise=0.5, seed=9)
    Vd = _cuda(V)
    lab, cent, seeds, r = H.spectral_cluster(Vd, c, synth.kmeans_first(n, 0))
    Xt = H.row_normalize(Vd)
    lab, cent, seeds, Xt = to_np(lab), to_np(cent), to_np(seeds), to_np(Xt)
    del Vd
    g = synth.rng(10)
    rows = g.choice(n, 4096, replace=False)
    X_rows = C.features(V[rows])                       # Step 4 is row-wise
    assert np.array_equal(_bits(Xt[:, rows].T), _bits(X_rows))
    assert r < 100 and len(set(seeds.tolist())) == c
    # nearest centroid within float32 rounding of the distance
    C32 = cent.astype(np.float32).astype(np.float64)
    d2 = ((X_rows.astype(np.float64)[:, None, :] - C32[None]) ** 2).sum(-1)
    mine = d2[np.arange(rows.size), lab[rows]]
    assert np.all(mine <= d2.min(axis=1) * (1 + 1e-5) + 1e-12)
    # each centroid the float64 mean of its members (fixed-point error <= 2^-37)
    X = Xt.T.astype(np.float64)
    cnt = np.bincount(lab, minlength=c)
    assert cnt.min() > 0
    for d in range(0, c, 7):
        means = np.bincount(lab, weights=X[:, d], minlength=c) / cnt
        assert np.max(np.abs(means - cent[:, d])) < 2.0 ** -36
    assert C.adjusted_rand_index(lab, truth) == 1.0


def test_gpu_solve_then_cluster_recovers_sbm(H):
    g = synth.sbm_edges(20000, 20, d_in=16.0, d_out=2.0, seed=2)
    A = device_csr(H, g)
    ev, V, info = H.solve(A, 20, 10, 11, 60, 1e-8)
    assert info.status == 0
    lab, _, _, r = H.spectral_cluster(V, 20, synth.kmeans_first(g.n, 0))
    assert C.adjusted_rand_index(to_np(lab), g.labels) == 1.0
    assert C.normalized_mutual_info(to_np(lab), g.labels) == pytest.approx(1.0, abs=1e-12)
