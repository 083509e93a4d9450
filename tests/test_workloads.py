"""Properties of the second workload family's generators (synth): the MAWI stand-in (connected,
ultra-sparse, degree-1 majority, giant hubs) and the degree-corrected SBM stand-ins of the
Graph Challenge categories (average degree, share of edges between blocks, block size
variation), plus determinism.  The paper's own graphs are not reproduced."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph

import synth


def _degrees(g):
    return np.bincount(g.src, minlength=g.n) + np.bincount(g.dst, minlength=g.n)


def _simple(g):
    assert np.all(g.src != g.dst)
    keys = np.minimum(g.src, g.dst).astype(np.int64) * g.n + np.maximum(g.src, g.dst)
    assert np.unique(keys).size == keys.size


def test_powerlaw_graph_shape():
    n = 200_000
    g = synth.powerlaw_tree_edges(n, 3.0, seed=9)
    _simple(g)
    d = _degrees(g)
    A = sp.coo_matrix((np.ones(g.src.size), (g.src, g.dst)), shape=(n, n))
    assert csgraph.connected_components(A, directed=False)[0] == 1
    assert abs(2 * g.src.size / n - 3.0) < 0.01            # average degree 3.0
    assert (d == 1).mean() > 0.6                           # most nodes are leaves
    assert d.max() > n / (2 * np.log(n))                   # a giant hub (about n / ln n)
    assert np.array_equal(synth.powerlaw_tree_edges(n, 3.0, seed=9).src, g.src)


@pytest.mark.parametrize("cat", ["lbolbsv", "lbohbsv", "hbolbsv", "hbohbsv"])
def test_dcsbm_categories(cat):
    w = synth.workload(f"dcsbm5m_{cat}@100000")
    g = w["graph"]
    _simple(g)
    assert abs(2 * g.src.size / g.n - 48.5) < 0.02 * 48.5   # avg degree (repeats removed)
    between = (g.labels[g.src] != g.labels[g.dst]).mean()
    want = 0.2 if cat.startswith("lbo") else 0.45
    assert abs(between - want) < 0.015
    sizes = np.bincount(g.labels, minlength=64)
    assert sizes.sum() == g.n and np.all(np.diff(g.labels) >= 0)
    if cat.endswith("lbsv"):
        assert sizes.max() / sizes.min() < 1.6
    else:
        assert sizes.max() / sizes.min() > 10
    assert w["k"] == 64 and np.unique(g.labels).size == 64


def test_knn_gmm_exact_neighbours():
    """The kNN-GMM workload (Gaussian mixture in 16-D, 10 nearest neighbours): every node's
    out-edges are exactly its 10 nearest other points by float64 Euclidean distance (ties to the
    lower index), checked by brute force; the graph the Laplacian is built from is their
    symmetrisation (an undirected edge wherever either end lists the other)."""
    n, dim, knn = 3000, 16, 10
    g = synth.knn_gmm_edges(n, dim=dim, n_comp=50, knn=knn, seed=3)
    # the generator's points, redrawn from the same seeded stream
    r = synth.rng(3)
    means = r.uniform(-10.0, 10.0, (50, dim))
    comp = r.integers(0, 50, n)
    x = means[comp] + r.standard_normal((n, dim))
    assert np.array_equal(g.labels, comp)
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    want = np.argsort(d2, axis=1, kind="stable")[:, :knn]
    assert np.all(g.src != g.dst)
    assert np.all(np.bincount(g.src, minlength=n) == knn)
    order = np.lexsort((g.dst, g.src))
    got = g.dst[order].reshape(n, knn)
    assert np.array_equal(np.sort(got, axis=1), np.sort(want, axis=1))
    # symmetrised degree: at least knn per node, at most knn + in-degree
    A = sp.coo_matrix((np.ones(g.src.size), (g.src, g.dst)), shape=(n, n)).tocsr()
    S = ((A + A.T) > 0).astype(np.int8)
    deg = np.asarray(S.sum(axis=1)).ravel()
    assert deg.min() >= knn and deg.max() <= knn + np.bincount(g.dst, minlength=n).max()
    assert S.diagonal().sum() == 0
    g2 = synth.knn_gmm_edges(n, dim=dim, n_comp=50, knn=knn, seed=3)
    assert np.array_equal(g2.src, g.src) and np.array_equal(g2.dst, g.dst)


def test_knn_gmm_reduced_workload_components():
    """The 200,000-point reduction of the kNN-GMM workload has one connected component per
    mixture component (50), so lambda = 0 has multiplicity 50 = k.  The oracle goldens record
    what Algorithm 2 finds there: from k Gaussian start columns it returns all 50 null
    directions; from k_b = 10 it returns fewer, because the filter is the identity on the null
    space (p(0) = 1) and only rounding noise brings null directions beyond the span of the
    start block into the basis (locking then skips copies of the multiple eigenvalue)."""
    import json
    import os
    w = synth.workload("knn2m@200000")
    g = w["graph"]
    n = g.n
    A = sp.coo_matrix((np.ones(g.src.size), (g.src, g.dst)), shape=(n, n))
    ncomp, lab = csgraph.connected_components(A, directed=False)
    assert ncomp == 50
    # components never mix mixture components
    assert np.all(np.bincount(lab, minlength=ncomp) > 0)
    assert all(np.unique(g.labels[lab == c]).size == 1 for c in range(ncomp))
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

    def zeros(name):
        with open(os.path.join(here, name)) as f:
            gold = json.load(f)
        return int(np.sum(np.abs(np.asarray(gold["evals"])) < 1e-10)), gold

    z_k, gk = zeros("oracle_knn2m@200000_v0k.json")
    z_b, gb = zeros("oracle_knn2m@200000.json")
    assert gk["v0_cols"] == 50 and z_k == ncomp
    assert z_b < ncomp
