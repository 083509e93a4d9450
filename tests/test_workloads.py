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
