"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds no arithmetic of the eigensolver: it only draws graphs (as
undirected edge lists of int32 node pairs) and random starting blocks.  Every
draw goes through numpy's Philox bit generator with an explicit seed, so the
same call returns the same bytes on x86 and Arm hosts.

Graph families (stand-ins for the workloads the paper evaluates on, Sec. 4):

* ``sbm_edges``       stochastic block model (HPEC Graph Challenge style
                      partitions, Sec. 4.1) with equal planted clusters;
* ``batch_sbm``       many SBM graphs of log-uniform size;
* ``knn_gmm_edges``   symmetrised k-nearest-neighbour graph of a Gaussian
                      mixture;
* ``rmat_edges``      R-MAT power-law graph (Graph500 style, Table 2);
* closed-form graphs (cycle, path, hypercube, complete, complete bipartite,
  star, disjoint unions) whose Laplacian spectra are known exactly.

Edge lists may contain duplicates, both orientations and self loops; the
Laplacian builders on either side are specified to symmetrise, deduplicate and
drop self loops.  ``reattach_isolated`` implements the "isolated nodes are
reattached by one random edge" rule of the SBM workloads.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "rng",
    "gaussian_block",
    "sbm_edges",
    "reattach_isolated",
    "batch_sbm",
    "knn_gmm_edges",
    "rmat_edges",
    "cycle_edges",
    "path_edges",
    "hypercube_edges",
    "complete_edges",
    "complete_bipartite_edges",
    "star_edges",
    "disjoint_union",
    "Graph",
    "workload",
]


def rng(seed: int) -> np.random.Generator:
    """Philox-backed generator; the only source of randomness in this module."""
    return np.random.Generator(np.random.Philox(int(seed)))


def gaussian_block(n: int, cols: int, seed: int = 0) -> np.ndarray:
    """Row-major n x cols float64 block of standard normal numbers (the V0 block)."""
    return rng(seed).standard_normal((n, cols))


def gnn_random_features(n: int, d_r: int, seed: int) -> np.ndarray:
    """Row-major n x d_r float32 standard normal node features (the network's random inputs)."""
    return rng(seed).standard_normal((n, d_r)).astype(np.float32)


def kmeans_first(n: int, seed: int) -> int:
    """Index of the first k-means seed: one uniform draw from [0, n)."""
    return int(rng(seed).integers(0, n))


def planted_embedding(n: int, c: int, dim: int, noise: float = 0.05, seed: int = 0,
                      contiguous: bool = True):
    """Block shaped like the k leading eigenvectors of a c-cluster graph: row i is
    q_{label_i} / sqrt(n_{label_i}) plus isotropic Gaussian noise whose expected length is about
    `noise` times that row's length, q_j orthonormal directions in R^dim (dim >= c).  Labels are cluster-contiguous (as the SBM
    numbers its nodes) or shuffled.  Returns (V float64 n x dim, labels int32)."""
    g = rng(seed)
    sizes = np.full(c, n // c, dtype=np.int64)
    sizes[: n % c] += 1
    labels = np.repeat(np.arange(c, dtype=np.int32), sizes)
    if not contiguous:
        labels = labels[g.permutation(n)]
    Q, _ = np.linalg.qr(g.standard_normal((dim, c)))
    scale = 1.0 / np.sqrt(sizes[labels].astype(np.float64))
    V = Q.T[labels] * scale[:, None]
    V += g.standard_normal((n, dim)) * (noise / np.sqrt(dim) * scale)[:, None]
    return V, labels


def gnn_init(d_in: int, width: int, k: int, layers: int = 3, seed: int = 0) -> np.ndarray:
    """Flat float32 initial parameters of the start-block network: every weight matrix
    (fan_in x fan_out) normal with standard deviation sqrt(1 / fan_in), biases zero, in the
    order W_1, U_1, b_1, ..., W_L, U_L, b_L, Wo."""
    g = rng(seed)
    parts = []
    p = d_in
    for _ in range(layers):
        parts.append(g.standard_normal(p * width) * np.sqrt(1.0 / p))
        parts.append(g.standard_normal(p * width) * np.sqrt(1.0 / p))
        parts.append(np.zeros(width))
        p = width
    parts.append(g.standard_normal(width * k) * np.sqrt(1.0 / width))
    return np.concatenate(parts).astype(np.float32)


@dataclass
class Graph:
    """An undirected graph on nodes 0..n-1 given as an edge list."""

    n: int
    src: np.ndarray  # int32
    dst: np.ndarray  # int32
    name: str = ""
    labels: np.ndarray | None = None  # planted cluster of each node, if any

    @property
    def n_edges(self) -> int:
        return int(self.src.shape[0])


def _as_graph(n, src, dst, name, labels=None) -> Graph:
    return Graph(int(n), np.ascontiguousarray(src, dtype=np.int32),
                 np.ascontiguousarray(dst, dtype=np.int32), name, labels)


# ----------------------------------------------------------------------------
# closed-form families
# ----------------------------------------------------------------------------

def cycle_edges(n: int) -> Graph:
    i = np.arange(n, dtype=np.int64)
    return _as_graph(n, i, (i + 1) % n, f"cycle{n}")


def path_edges(n: int) -> Graph:
    i = np.arange(n - 1, dtype=np.int64)
    return _as_graph(n, i, i + 1, f"path{n}")


def hypercube_edges(d: int) -> Graph:
    n = 1 << d
    i = np.arange(n, dtype=np.int64)
    src = np.concatenate([i for _ in range(d)])
    dst = np.concatenate([i ^ (1 << t) for t in range(d)])
    keep = src < dst
    return _as_graph(n, src[keep], dst[keep], f"hypercube{d}")


def complete_edges(n: int) -> Graph:
    iu = np.triu_indices(n, 1)
    return _as_graph(n, iu[0], iu[1], f"K{n}")


def complete_bipartite_edges(a: int, b: int) -> Graph:
    u = np.repeat(np.arange(a), b)
    v = np.tile(np.arange(b), a) + a
    return _as_graph(a + b, u, v, f"K{a},{b}")


def star_edges(leaves: int) -> Graph:
    v = np.arange(1, leaves + 1)
    return _as_graph(leaves + 1, np.zeros_like(v), v, f"star{leaves}")


def disjoint_union(*graphs: Graph) -> Graph:
    off = 0
    src, dst = [], []
    for g in graphs:
        src.append(g.src.astype(np.int64) + off)
        dst.append(g.dst.astype(np.int64) + off)
        off += g.n
    return _as_graph(off, np.concatenate(src), np.concatenate(dst),
                     "+".join(g.name for g in graphs))


# ----------------------------------------------------------------------------
# random families
# ----------------------------------------------------------------------------

def _sorted_unique(x: np.ndarray) -> np.ndarray:
    """np.unique of an int64 array (sorted distinct values), by sorting."""
    x = np.sort(x, kind="stable")
    if x.shape[0] == 0:
        return x
    keep = np.empty(x.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(x[1:], x[:-1], out=keep[1:])
    return x[keep]


def _unique_pairs(u: np.ndarray, v: np.ndarray, n: int) -> np.ndarray:
    lo = np.minimum(u, v).astype(np.int64)
    hi = np.maximum(u, v).astype(np.int64)
    return _sorted_unique(lo * n + hi)


def _sample_pairs(g, k, draw, n):
    """k distinct unordered pairs drawn uniformly by rejection from ``draw``."""
    keys = np.empty(0, dtype=np.int64)
    while keys.shape[0] < k:
        need = k - keys.shape[0]
        m = int(need * 1.1) + 16
        u, v = draw(m)
        ok = u != v
        new = _unique_pairs(u[ok], v[ok], n)
        keys = _sorted_unique(np.concatenate([keys, new]))
        if keys.shape[0] > k:
            keys = g.permutation(keys)[:k]
            keys.sort()
    return keys


def sbm_edges(n: int, c: int, *, p_in: float | None = None, p_out: float | None = None,
              d_in: float | None = None, d_out: float | None = None, seed: int = 1,
              reattach: bool = True) -> Graph:
    """Stochastic block model on n nodes with c planted clusters.

    Cluster sizes are floor(n/c) with the first n mod c clusters one larger;
    node ids are cluster-contiguous.  Each unordered pair is an edge
    independently with probability p_in (same cluster) or p_out (different
    clusters); the edge count of each population is drawn Binomial and the
    pairs uniformly without replacement, which is the same distribution.
    Expected degrees may be given instead: p_in = d_in/(n_c - 1),
    p_out = d_out/(n - n_c) with n_c the mean cluster size.
    """
    g = rng(seed)
    sizes = np.full(c, n // c, dtype=np.int64)
    sizes[: n % c] += 1
    starts = np.concatenate([[0], np.cumsum(sizes)])
    labels = np.repeat(np.arange(c, dtype=np.int32), sizes)
    nc = n / c
    if p_in is None:
        p_in = d_in / (nc - 1.0)
    if p_out is None:
        p_out = d_out / (n - nc)
    keys = []
    for a in range(c):
        s, sz = int(starts[a]), int(sizes[a])
        m_pairs = sz * (sz - 1) // 2
        k = int(g.binomial(m_pairs, p_in)) if m_pairs > 0 else 0
        if k > 0:
            draw = lambda m, s=s, sz=sz: (g.integers(s, s + sz, m), g.integers(s, s + sz, m))
            keys.append(_sample_pairs(g, k, draw, n))
    m_out = (n * (n - 1)) // 2 - int(np.sum(sizes * (sizes - 1) // 2))
    k_out = int(g.binomial(m_out, p_out)) if m_out > 0 else 0
    if k_out > 0:
        def draw_out(m):
            u = g.integers(0, n, m)
            v = g.integers(0, n, m)
            same = labels[u] == labels[v]
            return u[~same], v[~same]
        keys.append(_sample_pairs(g, k_out, draw_out, n))
    keys = np.concatenate(keys) if keys else np.empty(0, dtype=np.int64)
    src, dst = keys // n, keys % n
    if reattach:
        src, dst = reattach_isolated(n, src, dst, g)
    return _as_graph(n, src, dst, f"sbm{n}c{c}", labels)


def reattach_isolated(n: int, src: np.ndarray, dst: np.ndarray, g: np.random.Generator):
    """Give every node with no neighbour (self loops ignored) one random edge.

    The isolated set is computed once; each isolated node, in increasing id
    order, draws its partner uniformly from the other n - 1 nodes.
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    ok = src != dst
    deg = np.bincount(src[ok], minlength=n) + np.bincount(dst[ok], minlength=n)
    iso = np.flatnonzero(deg == 0)
    if iso.size == 0 or n < 2:
        return src, dst
    j = g.integers(0, n - 1, iso.size)
    j = j + (j >= iso)  # uniform over [0, n) \ {i}
    return np.concatenate([src, iso]), np.concatenate([dst, j])


def batch_sbm(n_graphs: int = 512, n_lo: int = 2000, n_hi: int = 200000, c_lo: int = 4,
              c_hi: int = 32, d_in: float = 12.0, d_out: float = 1.5, seed: int = 4,
              base_seed: int = 1000):
    """Many independent SBM graphs: sizes log-uniform in [n_lo, n_hi], c uniform."""
    g = rng(seed)
    ns = np.floor(np.exp(g.uniform(math.log(n_lo), math.log(n_hi), n_graphs))).astype(np.int64)
    cs = g.integers(c_lo, c_hi + 1, n_graphs)
    return [sbm_edges(int(ns[i]), int(cs[i]), d_in=d_in, d_out=d_out, seed=base_seed + i)
            for i in range(n_graphs)]


def knn_gmm_edges(n: int, dim: int = 16, n_comp: int = 50, knn: int = 10, seed: int = 3,
                  box: float = 10.0) -> Graph:
    """Symmetrised, unweighted k-NN graph of points from an isotropic Gaussian mixture.

    Component means are uniform in [-box, box]^dim, unit variance, uniform
    weights; points stay in draw order.  Neighbours are exact Euclidean
    nearest neighbours (ties to the lower index), found with a KD-tree.
    """
    from scipy.spatial import cKDTree

    g = rng(seed)
    means = g.uniform(-box, box, (n_comp, dim))
    comp = g.integers(0, n_comp, n)
    x = means[comp] + g.standard_normal((n, dim))
    tree = cKDTree(x)
    _, idx = tree.query(x, k=knn + 1, workers=-1)
    src = np.repeat(np.arange(n, dtype=np.int64), knn + 1)
    dst = idx.reshape(-1).astype(np.int64)
    keep = src != dst
    return _as_graph(n, src[keep], dst[keep], f"knn{n}", comp.astype(np.int32))


def powerlaw_tree_edges(n: int, avg_deg: float = 3.0, seed: int = 9) -> Graph:
    """Ultra-sparse power-law graph with giant hubs, connected (stand-in for the MAWI traffic
    graph of Table 2: N = 18M, average degree 3.0, heavy row imbalance).

    Node weights w_j = 1/(j + 1) (Zipf).  A random recursive tree: node i >= 1 joins one
    earlier node j < i drawn with probability w_j / sum_{l<i} w_l; then Chung-Lu edges, both
    endpoints drawn with probability proportional to w, self loops and repeats removed, in up
    to four rounds until the graph has n * avg_deg / 2 edges.  Node ids are permuted uniformly
    at random at the end.
    Most nodes end with degree 1 (leaves of hubs); the largest hub holds about n / ln n."""
    g = rng(seed)
    w = 1.0 / (np.arange(n, dtype=np.float64) + 1.0)
    C = np.cumsum(w)
    i = np.arange(1, n, dtype=np.int64)
    parent = np.minimum(np.searchsorted(C, g.random(n - 1) * C[i - 1], side="right"), i - 1)
    target = int(round(n * avg_deg / 2))
    keys = _unique_pairs(i, parent, n)
    for _ in range(4):                       # Chung-Lu edges until the target count is met
        m_extra = target - keys.size
        if m_extra <= 0:
            break
        q = np.sort(g.random(2 * m_extra)) * C[-1]      # sorted queries: cache-friendly search
        ends = np.minimum(np.searchsorted(C, q, side="right"), n - 1)
        ends = ends[g.permutation(ends.size)]
        u, v = ends[:m_extra], ends[m_extra:]
        keep = u != v
        keys = _sorted_unique(np.concatenate([keys, _unique_pairs(u[keep], v[keep], n)]))
    perm = g.permutation(n).astype(np.int64)
    return _as_graph(n, perm[keys // n], perm[keys % n], f"powerlaw{n}")


def dcsbm_edges(n: int, c: int, avg_deg: float, between: float, size_var: str = "low",
                seed: int = 10) -> Graph:
    """Degree-corrected SBM with block overlap and block size variation (stand-in for the
    HPEC Graph Challenge partition graphs of Sec. 4.1, LBO/HBO x LBSV/HBSV; Table 2 lists
    5M- and 20M-node ones with average degree 48.5).

    Block sizes: n times Dirichlet(200) proportions ("low" variation) or Dirichlet(1) ("high");
    node ids block-contiguous (labels = block).  Degree weights theta_i: Pareto with tail
    exponent 2.5, capped at 10.  Each edge draw: first endpoint u with probability proportional
    to theta; with probability 1 - `between` the second endpoint v proportional to theta inside
    u's block, else proportional to theta outside it.  Drawn as multinomial counts per node (the
    same distribution as independent draws, in O(n + m)): first endpoints per node, second
    endpoints per block, paired by a random permutation; outside-block endpoints drawn over all
    nodes and redrawn while in u's block.  Self loops and repeats are removed and more edges
    drawn, in up to four rounds, until the graph has n * avg_deg / 2 edges."""
    g = rng(seed)
    alpha = 200.0 if size_var == "low" else 1.0
    sizes = np.maximum(1, np.round(g.dirichlet(np.full(c, alpha)) * n)).astype(np.int64)
    sizes[int(np.argmax(sizes))] += n - int(sizes.sum())
    labels = np.repeat(np.arange(c, dtype=np.int32), sizes)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    theta = np.minimum((1.0 - g.random(n)) ** (-1.0 / 1.5), 10.0)
    p_all = theta / theta.sum()

    def draw(m):
        u = np.repeat(np.arange(n, dtype=np.int64), g.multinomial(m, p_all))
        bu = labels[u]
        within = g.random(m) >= between
        v = np.empty(m, dtype=np.int64)
        e_start = np.searchsorted(bu, np.arange(c + 1))   # u is sorted, so by block
        for b in range(c):
            idx = e_start[b] + np.flatnonzero(within[e_start[b]:e_start[b + 1]])
            if idx.size == 0:
                continue
            s0, s1 = int(starts[b]), int(starts[b + 1])
            tb = theta[s0:s1]
            cnt = g.multinomial(idx.size, tb / tb.sum())
            v[idx] = np.repeat(np.arange(s0, s1, dtype=np.int64), cnt)[g.permutation(idx.size)]
        idx = np.flatnonzero(~within)
        while idx.size:
            vv = np.repeat(np.arange(n, dtype=np.int64), g.multinomial(idx.size, p_all))
            vv = vv[g.permutation(idx.size)]
            v[idx] = vv
            idx = idx[labels[vv] == bu[idx]]
        keep = u != v
        return _unique_pairs(u[keep], v[keep], n)

    target = int(round(n * avg_deg / 2))
    keys = draw(target)
    for _ in range(3):
        if keys.size >= target:
            break
        keys = _sorted_unique(np.concatenate([keys, draw(target - keys.size)]))
    return _as_graph(n, keys // n, keys % n, f"dcsbm{n}c{c}", labels)


def _rmat_level_tables(probs: np.ndarray, levels: int):
    """Tables mapping a 16-bit uniform to the i- and j-bits of `levels` consecutive R-MAT
    levels (bit t = level t of the group).  The outcome probabilities (products of the
    quadrant probabilities) are quantised to multiples of 2^-16."""
    p = np.ones(1)
    for _ in range(levels):
        p = np.outer(p, probs).ravel()          # outcome index: q_0 * 4^(levels-1) + ... + q_last
    edges = np.round(np.cumsum(p) * 65536.0).astype(np.int64)
    edges[-1] = 65536
    outcome = np.searchsorted(edges, np.arange(65536), side="right")
    ti = np.zeros(65536, dtype=np.uint32)
    tj = np.zeros(65536, dtype=np.uint32)
    for t in range(levels):
        q = (outcome // 4 ** (levels - 1 - t)) % 4  # quadrant of level t: (i, j) = (q >> 1, q & 1)
        ti |= ((q >> 1) & 1).astype(np.uint32) << t
        tj |= (q & 1).astype(np.uint32) << t
    return ti, tj


def rmat_edges(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
               c: float = 0.19, seed: int = 5, chunk: int = 1 << 22) -> Graph:
    """R-MAT sampler (Graph500 parameters by default), no vertex permutation.

    edge_factor * 2^scale directed samples; each picks one quadrant per level with
    probabilities (a, b, c, 1-a-b-c) for (i, j) bits (0,0), (0,1), (1,0), (1,1).  Levels are
    drawn two at a time from one 16-bit uniform through a table of the 16 joint outcomes (their
    probabilities quantised to multiples of 2^-16: at most 0.3% relative for the rarest, d*d).
    """
    n = 1 << scale
    m = edge_factor * n
    g = rng(seed)
    probs = np.array([a, b, c, 1.0 - a - b - c])
    t2i, t2j = _rmat_level_tables(probs, 2)
    t1i, t1j = _rmat_level_tables(probs, 1)
    pairs, odd = divmod(scale, 2)
    words = (pairs + odd + 3) // 4               # 64-bit draws per edge (four 16-bit uniforms)
    srcs, dsts = [], []
    for lo in range(0, m, chunk):
        k = min(chunk, m - lo)
        raw = g.bit_generator.random_raw(k * words).reshape(k, words)
        u16 = raw.view(np.uint16)                # k x (4 words)
        u = np.zeros(k, dtype=np.uint32)
        v = np.zeros(k, dtype=np.uint32)
        for t in range(pairs):
            r = u16[:, t]
            u |= t2i[r] << np.uint32(2 * t)
            v |= t2j[r] << np.uint32(2 * t)
        if odd:
            r = u16[:, pairs]
            u |= t1i[r] << np.uint32(2 * pairs)
            v |= t1j[r] << np.uint32(2 * pairs)
        srcs.append(u.astype(np.int64))
        dsts.append(v.astype(np.int64))
    src = np.concatenate(srcs)
    dst = np.concatenate(dsts)
    src, dst = reattach_isolated(n, src, dst, g)
    return _as_graph(n, src, dst, f"rmat{scale}")


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def workload(name: str) -> dict:
    """Graph plus solver parameters of the named benchmark workloads.

    sbm10k   : SBM N=10,000, 10 clusters, p_in=1e-3, p_out=2e-5, k=10, b=5, m=11, act_max=30
    sbm1m    : SBM N=1,000,000, 100 clusters, d_in=16, d_out=2, k=100, b=20, m=15, act_max=300
    sbm1m_comb: the same graph's combinatorial Laplacian D - S, bounds by 20-step Lanczos
    dcsbm5m_{lbo|hbo}{lbsv|hbsv}: degree-corrected SBM N=5,000,000, 64 blocks, average degree
              48.5, 20% (LBO) or 45% (HBO) of edges between blocks, block sizes Dirichlet(200)
              (LBSV) or Dirichlet(1) (HBSV); k=64, b=16, m=11, act_max=192
    mawi18m  : connected power-law graph N=18,000,000, average degree 3.0 (Zipf-weighted random
              recursive tree plus Chung-Lu edges); k=16, b=8, m=15, act_max=96
    knn2m    : kNN-GMM 2,000,000 x 16-D, 50 components, 10-NN, k=50, b=10, m=13, act_max=150
    rmat24   : R-MAT scale 24, ef 16, k=64, b=16, m=15, act_max=192
    Scaled-down variants (for tests) take a suffix, e.g. ``sbm1m@50000`` keeps
    the per-node statistics with fewer nodes.
    """
    base, _, size = name.partition("@")
    tol = 1e-8
    if base == "sbm10k":
        n = int(size) if size else 10000
        gr = sbm_edges(n, 10, p_in=1e-3 * 10000 / n, p_out=2e-5 * 10000 / n, seed=1)
        return dict(graph=gr, k=10, b=5, m=11, act_max=30, tol=tol, v0_seed=0,
                    desc=f"SBM N={n} c=10 p_in=1e-3 p_out=2e-5")
    if base in ("sbm1m", "sbm1m_comb"):
        n = int(size) if size else 1000000
        c = 100 if n >= 100000 else max(4, n // 10000)
        gr = sbm_edges(n, c, d_in=16.0, d_out=2.0, seed=2)
        if base == "sbm1m_comb":
            return dict(graph=gr, k=c, b=20, m=15, act_max=300, tol=tol, v0_seed=0,
                        kind="combinatorial", bounds="lanczos", lanczos_steps=20,
                        desc=f"combinatorial Laplacian D - S of the SBM N={n} c={c} d_in=16 "
                             f"d_out=2, bounds by 20-step Lanczos")
        return dict(graph=gr, k=c, b=20, m=15, act_max=300, tol=tol, v0_seed=0,
                    desc=f"SBM N={n} c={c} d_in=16 d_out=2")
    if base.startswith("dcsbm5m_") and base[8:] in ("lbolbsv", "lbohbsv", "hbolbsv", "hbohbsv"):
        n = int(size) if size else 5000000
        cat = base[8:]
        between = 0.2 if cat.startswith("lbo") else 0.45
        var = "low" if cat.endswith("lbsv") else "high"
        gr = dcsbm_edges(n, 64, 48.5, between, var, seed=10)
        return dict(graph=gr, k=64, b=16, m=11, act_max=192, tol=tol, v0_seed=0,
                    desc=f"degree-corrected SBM N={n}, 64 blocks, avg degree 48.5, "
                         f"{int(between * 100)}% of edges between blocks, {var} block size "
                         f"variation ({cat.upper()} stand-in)")
    if base == "mawi18m":
        n = int(size) if size else 18000000
        gr = powerlaw_tree_edges(n, 3.0, seed=9)
        return dict(graph=gr, k=16, b=8, m=15, act_max=96, tol=tol, v0_seed=0,
                    desc=f"connected power-law graph N={n}, avg degree 3.0, Zipf hubs "
                         f"(MAWI stand-in)")
    if base == "knn2m":
        n = int(size) if size else 2000000
        gr = knn_gmm_edges(n, seed=3)
        return dict(graph=gr, k=50, b=10, m=13, act_max=150, tol=tol, v0_seed=0,
                    desc=f"kNN graph of {n} points, 16-D 50-component Gaussian mixture, 10-NN")
    if base == "rmat24":
        scale = int(size) if size else 24
        gr = rmat_edges(scale, seed=5)
        return dict(graph=gr, k=64, b=16, m=15, act_max=192, tol=tol, v0_seed=0,
                    desc=f"R-MAT scale {scale} edge factor 16 (0.57, 0.19, 0.19, 0.05)")
    raise KeyError(name)
