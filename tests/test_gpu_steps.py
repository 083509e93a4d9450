"""Parity of each single step of the CUDA path with the oracle (through the C-ABI).

Eq. (1) Laplacian assembly (bit-exact), Eq. (6) SpMM, Algorithm 3 filter
(float64 and float32 recurrence), Step 6 orthonormalisation, Step 9 eigh.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import device_csr, oracle_csr, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import paper_2212_04443_gb300 as P
    return P.Handle()


GRAPHS = [
    lambda: synth.cycle_edges(97),
    lambda: synth.path_edges(50),
    lambda: synth.sbm_edges(3000, 7, d_in=9, d_out=1.5, seed=5),
    lambda: synth.sbm_edges(2500, 5, p_in=1e-3, p_out=1e-4, seed=6, reattach=False),  # isolated
    lambda: synth.disjoint_union(synth.complete_edges(70), synth.star_edges(5000)),     # long row
    lambda: synth.rmat_edges(12, seed=9),
]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_laplacian_bit_exact(H, gi):
    g = GRAPHS[gi]()
    # add duplicates, reversed copies and self loops: the builder must fold them
    rng = synth.rng(100 + gi)
    extra = rng.integers(0, g.n, 64)
    src = np.concatenate([g.src, g.dst[:50], extra]).astype(np.int32)
    dst = np.concatenate([g.dst, g.src[:50], extra]).astype(np.int32)
    g2 = synth.Graph(g.n, src, dst)
    A = device_csr(H, g2)
    L = oracle_csr(g2)
    assert np.array_equal(to_np(A.rowptr), L.rowptr)
    assert np.array_equal(to_np(A.colidx), L.colidx)
    assert np.array_equal(to_np(A.val).view(np.uint64), L.val.view(np.uint64))
    assert np.array_equal(to_np(A.val_f32), L.val.astype(np.float32))
    assert H.check_csr(A) == 0


def test_laplacian_rejects_out_of_range(H):
    import torch
    import paper_2212_04443_gb300 as P
    src = torch.tensor([0, 1, 5], dtype=torch.int32, device="cuda")
    dst = torch.tensor([1, 2, 0], dtype=torch.int32, device="cuda")
    with pytest.raises(P.BchdavError) as ei:
        H.build_laplacian(5, src, dst)
    assert ei.value.status == -1


def test_check_csr_flags_unsorted(H):
    import torch
    import paper_2212_04443_gb300 as P
    A = P.DeviceCSR(3, torch.tensor([0, 2, 3, 4], dtype=torch.int32, device="cuda"),
                    torch.tensor([1, 0, 1, 2], dtype=torch.int32, device="cuda"),
                    torch.ones(4, dtype=torch.float64, device="cuda"))
    assert H.check_csr(A) == -2


@pytest.mark.parametrize("b", [1, 5, 20, 33])
def test_spmm_matches_scipy(H, b):
    import torch
    g = synth.sbm_edges(20011, 9, d_in=11, d_out=2, seed=3)
    A = device_csr(H, g)
    L = oracle_csr(g)
    X = synth.gaussian_block(g.n, b, 1)
    Y = to_np(H.spmm(A, torch.from_numpy(X).cuda()))
    ref = L.scipy() @ X
    assert np.abs(Y - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("b", [4, 20, 64])
def test_spmm_dd_matches_float64(H, b):
    """The mixed path's double-float product (Steps 7 and 12): within 2^-44 of sum |a_ij x_j|
    per entry (the pair arithmetic keeps ~48 bits), far inside float64's reach of float32's."""
    import torch
    g = synth.sbm_edges(20011, 9, d_in=11, d_out=2, seed=3)
    A = device_csr(H, g)
    L = oracle_csr(g)
    X = synth.gaussian_block(g.n, b, 5)
    X[7] *= 1e-30                      # tiny and huge entries take the float64 split path
    X[11] *= 1e30
    Y = to_np(H.spmm_dd(A, torch.from_numpy(X).cuda()))
    S = L.scipy()
    ref = S @ X
    bound = abs(S) @ np.abs(X)
    assert np.all(np.abs(Y - ref) <= 2.0 ** -44 * bound)
    big = bound > 1e-200
    assert (np.abs(Y - ref)[big] / bound[big]).max() < 1e-12   # not a float32 product


def test_spmm_dd_rejects_what_the_mixed_path_keeps_in_float64(H):
    import torch
    import paper_2212_04443_gb300 as P
    g = synth.sbm_edges(3000, 4, d_in=8, d_out=1, seed=2)
    A = device_csr(H, g)
    with pytest.raises(P.BchdavError):          # width not a multiple of 4
        H.spmm_dd(A, torch.zeros((g.n, 6), dtype=torch.float64, device="cuda"))
    Ah = device_csr(H, _hub_graph())            # rows that need segments
    with pytest.raises(P.BchdavError):
        H.spmm_dd(Ah, torch.zeros((Ah.n, 8), dtype=torch.float64, device="cuda"))


def _hub_graph():
    """Rows far over the 1024-nonzero segment length (star hubs of 5000 and 2500 leaves, whose
    lengths are not multiples of it) next to power-law and short rows."""
    return synth.disjoint_union(synth.star_edges(5000), synth.rmat_edges(12, seed=9),
                                synth.star_edges(2500), synth.path_edges(40))


@pytest.mark.parametrize("b", [1, 3, 8, 20, 33])
def test_spmm_long_rows_match_scipy(H, b):
    """Segmented rows: error within the float64 bound for a sum of len(row) products."""
    import torch
    g = _hub_graph()
    A = device_csr(H, g)
    L = oracle_csr(g)
    assert np.diff(L.rowptr).max() > 4 * 1024
    X = synth.gaussian_block(g.n, b, 11)
    Y = to_np(H.spmm(A, torch.from_numpy(X).cuda()))
    S = L.scipy()
    ref = S @ X
    bound = abs(S) @ np.abs(X)
    lens = np.diff(L.rowptr)[:, None]
    assert np.all(np.abs(Y - ref) <= 2 * lens * 2.0 ** -53 * bound + 1e-300)


def test_filter_f32_long_rows(H):
    import torch
    import paper_2212_04443_gb300 as P
    g = _hub_graph()
    A = device_csr(H, g)
    L = oracle_csr(g)
    m, a, b = 11, 0.05, 16
    X = synth.gaussian_block(g.n, b, 12)
    Y = to_np(H.filter(A, torch.from_numpy(X).cuda(), m, a, 2.0, 0.0, precision=P.PREC_MIXED))
    Yd = to_np(H.filter(A, torch.from_numpy(X).cuda(), m, a, 2.0, 0.0))
    ref = oracle.chebyshev_filter(L.scipy(), X, m, a, 2.0, 0.0)
    assert np.abs(Yd - ref).max() <= 1e-12 * np.abs(ref).max()
    # float32 sums over hub rows of 5000 terms: a wider (length-proportional) bound
    assert np.abs(Y - ref).max() <= 5000 * m * 2.0 ** -24 * np.abs(ref).max()


@pytest.mark.parametrize("m,a,b", [(1, 0.3, 4), (11, 0.002, 5), (15, 0.55, 20), (13, 0.2, 10),
                                   (7, 1.1, 3)])
def test_filter_f64_matches_oracle(H, m, a, b):
    import torch
    g = synth.sbm_edges(30000, 12, d_in=14, d_out=2, seed=4)
    A = device_csr(H, g)
    L = oracle_csr(g)
    X = synth.gaussian_block(g.n, b, 2)
    Y = to_np(H.filter(A, torch.from_numpy(X).cuda(), m, a, 2.0, 0.0))
    ref = oracle.chebyshev_filter(L.scipy(), X, m, a, 2.0, 0.0)
    assert np.abs(Y - ref).max() <= 1e-12 * np.abs(ref).max()


def test_spmm_schedule_table_shared_by_class(H):
    """The filter SpMM's block size is timed once per matrix class (N and mean row length in
    half-octaves, block width, value size, long rows): a second graph of the same class takes
    the table's entry without the 12 timing launches, a graph of another class is timed."""
    import torch
    import paper_2212_04443_gb300 as P
    b, m = 13, 5          # a block width no other test filters with

    def launches(g):
        A = device_csr(H, g)
        X = torch.from_numpy(synth.gaussian_block(g.n, b, 1)).cuda()
        torch.cuda.synchronize()
        l0 = P.launch_count()
        H.filter(A, X, m, 0.1, 2.0, 0.0)
        torch.cuda.synchronize()
        return P.launch_count() - l0

    first = launches(synth.sbm_edges(6000, 8, d_in=12, d_out=1.5, seed=71))
    same = launches(synth.sbm_edges(6000, 8, d_in=12, d_out=1.5, seed=72))
    other = launches(synth.sbm_edges(90000, 8, d_in=12, d_out=1.5, seed=73))
    assert first - same == 12
    assert other - same == 12


def test_filter_on_exact_cycle_modes(H):
    import torch
    n, m, a = 1000, 15, 0.35
    g = synth.cycle_edges(n)
    A = device_csr(H, g)
    i = np.arange(n)
    js = [0, 1, 7, 40, 250, 500]
    V = np.stack([np.cos(2 * math.pi * j * i / n) for j in js], 1)
    lam = np.array([1 - math.cos(2 * math.pi * j / n) for j in js])
    Y = to_np(H.filter(A, torch.from_numpy(V).cuda(), m, a, 2.0, 0.0))
    p = oracle.filter_polynomial(lam, m, a, 2.0, 0.0)
    assert np.abs(Y - V * p).max() <= 1e-12 * max(1.0, np.abs(p).max())


@pytest.mark.parametrize("m,a,b", [(11, 0.01, 8), (15, 0.5, 20), (13, 0.2, 10), (15, 0.3, 16)])
def test_filter_f32_recurrence(H, m, a, b):
    """float32 recurrence: error bounded by float32 rounding propagated through m steps."""
    import torch
    import paper_2212_04443_gb300 as P
    g = synth.sbm_edges(40000, 10, d_in=15, d_out=2, seed=8)
    A = device_csr(H, g)
    L = oracle_csr(g)
    X = synth.gaussian_block(g.n, b, 3)
    Y = to_np(H.filter(A, torch.from_numpy(X).cuda(), m, a, 2.0, 0.0, precision=P.PREC_MIXED))
    ref = oracle.chebyshev_filter(L.scipy(), X, m, a, 2.0, 0.0)
    # per-step relative rounding 2^-24, amplified at most linearly in m by the bounded recurrence
    assert np.abs(Y - ref).max() <= 4 * m * 2.0 ** -24 * np.abs(ref).max() * 8


@pytest.mark.parametrize("n,k,b", [(5000, 0, 6), (5000, 40, 8), (20000, 300, 20), (777, 17, 33)])
def test_orthonormalize_matches_oracle(H, n, k, b):
    import torch
    V = np.linalg.qr(synth.gaussian_block(n, k, 1))[0] if k else np.zeros((n, 0))
    X = synth.gaussian_block(n, b, 2)
    X[:, 1] += 1e-3 * X[:, 0]
    Xd = torch.from_numpy(X.copy()).cuda()
    Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda() if k else None
    nrep, ctr = H.orthonormalize(Vd, Xd, seed=7)
    Q = to_np(Xd)
    Qo, nrep_o, ctr_o = oracle.dgks_orthonormalize(V, X, seed=7)
    assert nrep == nrep_o == 0 and ctr == ctr_o
    assert np.abs(Q.T @ Q - np.eye(b)).max() < 1e-13
    if k:
        assert np.abs(V.T @ Q).max() < 1e-13
    assert np.abs(Q - Qo).max() < 1e-10


def test_orthonormalize_replaces_dependent_columns_like_oracle(H):
    import torch
    n, k, b = 4000, 12, 6
    V = np.linalg.qr(synth.gaussian_block(n, k, 4))[0]
    X = synth.gaussian_block(n, b, 5)
    X[:, 2] = X[:, 0] * 2.0
    X[:, 4] = V[:, 3]
    X[:, 5] = 0.0
    Xd = torch.from_numpy(X.copy()).cuda()
    nrep, ctr = H.orthonormalize(torch.from_numpy(V).cuda(), Xd, seed=11, rep_counter=3)
    Qo, nrep_o, ctr_o = oracle.dgks_orthonormalize(V, X, seed=11, rep_counter=3)
    Q = to_np(Xd)
    assert (nrep, ctr) == (nrep_o, ctr_o) == (3, 6)
    assert np.abs(Q.T @ Q - np.eye(b)).max() < 1e-13
    assert np.abs(V.T @ Q).max() < 1e-13
    assert np.abs(Q - Qo).max() < 1e-10


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 150, 300])
def test_eigh_matches_lapack(H, n):
    import torch
    rng = synth.rng(n)
    M = rng.standard_normal((n, n))
    S = (M + M.T) / 2
    D, Y = H.eigh(torch.from_numpy(S).cuda())
    D, Y = to_np(D), to_np(Y)
    ref = np.linalg.eigvalsh(S)
    assert np.all(np.diff(D) >= 0)
    assert np.abs(D - ref).max() < 1e-13 * max(1.0, np.abs(ref).max()) * max(1, n) ** 0.5
    assert np.abs(Y.T @ Y - np.eye(n)).max() < 1e-13 * max(1, n)
    assert np.abs(S @ Y - Y * D).max() < 1e-13 * max(1.0, np.abs(ref).max()) * max(1, n)


def test_eigh_known_spectrum_with_repeats(H):
    import torch
    n = 90
    Q = np.linalg.qr(synth.gaussian_block(n, n, 9))[0]
    d = np.concatenate([np.zeros(10), np.full(30, 0.5), np.linspace(0.6, 2.0, 50)])
    S = (Q * d) @ Q.T
    S = (S + S.T) / 2
    D, Y = H.eigh(torch.from_numpy(S).cuda())
    D, Y = to_np(D), to_np(Y)
    assert np.abs(D - np.sort(d)).max() < 1e-13
    assert np.abs(Y.T @ Y - np.eye(n)).max() < 1e-12
    assert np.abs(S @ Y - Y * D).max() < 1e-12


@pytest.mark.parametrize("spacing", [0.0, 1e-13, 1e-9])
def test_eigh_tight_clusters(H, spacing):
    """Clusters of eigenvalues that the tridiagonal route treats together: exact repeats, a chain
    1e-13 apart (wider than the route accepts, 1e3 eps ||T||, so the Jacobi kernel behind it
    takes over on the device) and a chain 1e-9 apart (separate eigenvalues whose vectors are
    computed independently and orthogonalised by the Newton-Schulz step)."""
    import torch
    n = 150
    Q = np.linalg.qr(synth.gaussian_block(n, n, 21))[0]
    d = np.concatenate([0.3 + spacing * np.arange(25), np.linspace(0.5, 1.8, n - 25)])
    S = (Q * d) @ Q.T
    S = (S + S.T) / 2
    D, Y = H.eigh(torch.from_numpy(S).cuda())
    D, Y = to_np(D), to_np(Y)
    assert np.abs(D - np.sort(d)).max() < 1e-13
    assert np.abs(Y.T @ Y - np.eye(n)).max() < 1e-12
    assert np.abs(S @ Y - Y * D).max() < 1e-12


def test_eigh_diagonal_plus_border(H):
    """The shape Step 15 leaves for Step 9: diag(d) bordered by k_b new columns."""
    import torch
    n, b = 120, 20
    rng = synth.rng(77)
    S = np.diag(np.sort(rng.uniform(0, 2, n)))
    B = 1e-3 * rng.standard_normal((n, b))
    S[:, -b:] = B
    S[-b:, :] = B.T
    S[-b:, -b:] = (S[-b:, -b:] + S[-b:, -b:].T) / 2
    D, Y = H.eigh(torch.from_numpy(S).cuda())
    D, Y = to_np(D), to_np(Y)
    assert np.abs(D - np.linalg.eigvalsh(S)).max() < 1e-14 * 10
    assert np.abs(S @ Y - Y * D).max() < 1e-13


@pytest.mark.parametrize("n,k,nb", [(50000, 300, 240), (1001, 77, 45), (4000, 16, 16), (777, 448, 5),
                                    (130001, 96, 70)])
@pytest.mark.parametrize("path", [0, 1, 2])
def test_rotate_matches_float64(H, n, k, nb, path):
    """Step 11 product V(:, :nb) = V(:, :k) Y: float64-accurate slice product on tcgen05 with
    tensor-memory level sums (path 0) or on warp-level mma (path 2), and float64 FMA (path 1)."""
    import torch
    rng = synth.rng(n + k)
    V = rng.standard_normal((n, k)) / np.sqrt(n)
    V[3] = 0.0                                   # a zero row
    V[5, :] *= 1e-12                             # a tiny row (its own exponent)
    V[7, 1] = 1e3                                # wide range inside one row
    Y = np.linalg.qr(rng.standard_normal((k, k)))[0][:, :nb]
    ref = V @ Y
    Vd = torch.from_numpy(V.copy()).cuda()
    H.rotate(Vd, torch.from_numpy(np.ascontiguousarray(Y)).cuda(), nb, dense_path=path)
    out = to_np(Vd)
    assert np.array_equal(out[:, nb:], V[:, nb:])          # columns beyond nb untouched
    # error bound of the rounded 48-bit split of both operands (|x| < 2^E <= 2 max|x|):
    # per entry <= K (2^-49 2^E_i max|Y_j| + max|V_i| 2^-49 2^F_j) + dropped levels <= K 2^-46 ...
    bound = k * 2.0 ** -45 * np.abs(V).max(1)[:, None] * np.abs(Y).max(0)[None, :]
    assert np.all(np.abs(out[:, :nb] - ref) <= bound + 1e-300)
    assert np.abs(out[3, :nb]).max() == 0.0


@pytest.mark.parametrize("n,ka,kb", [(1000003, 300, 20), (5000, 77, 45), (3001, 1, 1), (70000, 340, 20),
                                     (200000, 130, 64), (1037, 129, 33)])
@pytest.mark.parametrize("path", [0, 1, 2])
def test_gram_matches_float64(H, n, ka, kb, path):
    """Steps 6/8 product A^T B with a reduction over n rows (pieces of 1024 rows when split):
    tcgen05 with tensor-memory level sums and an integer fold (path 0), float64 FMA (path 1),
    warp-level mma (path 2); ragged tiles in every dimension."""
    import torch
    rng = synth.rng(n + ka)
    A = rng.standard_normal((n, ka)) / np.sqrt(n)
    B = rng.standard_normal((n, kb))
    A[:, 0] *= 1e-9                      # a column far below the others
    ref = A.T @ B
    out = to_np(H.gram(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), dense_path=path))
    # rounded 48-bit split: |err_pq| <= n 2^-46 max|A_p| max|B_q| (+ float64 summation)
    bound = n * 2.0 ** -45 * np.abs(A).max(0)[:, None] * np.abs(B).max(0)[None, :]
    assert np.all(np.abs(out - ref) <= bound + 1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("path", [0, 1, 2])
def test_gram_per_chunk_precision_with_hub_entries(H, path):
    """A^T B where one row dwarfs the rest of its column (a hub vertex).  The split scales each
    1024-row chunk by its own column exponent: with the hub alone in its chunk, the other rows
    keep their 48 bits.  One exponent for the whole column (2^21) would round every other entry
    to 2^-27 and leave an error near sqrt(n) 2^-28 ~ 1e-6 in that column of the product."""
    import torch
    n, ka, kb = 70001, 40, 12
    rng = synth.rng(77)
    A = rng.standard_normal((n, ka))
    B = rng.standard_normal((n, kb))
    A[:1024, 2] = 0.0
    A[17, 2] = 2.0 ** 20
    ref = A.T @ B
    out = to_np(H.gram(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), dense_path=path))
    fp = 4 * n * 2.0 ** -53 * (np.abs(A).T @ np.abs(B))     # float64 summation of either side
    err = np.abs(out - ref)
    ch = 1024
    bound = np.zeros((ka, kb))
    for r0 in range(0, n, ch):
        a = np.abs(A[r0:r0 + ch]).max(0)
        b = np.abs(B[r0:r0 + ch]).max(0)
        bound += min(ch, n - r0) * 2.0 ** -45 * a[:, None] * b[None, :]
    assert np.all(err <= bound + fp)
    assert np.all(err[2] <= 1e-3 * np.sqrt(n) * 2.0 ** -28 + fp[2])


def test_tcgen05_wait_timeout_reports_and_recovers(H, monkeypatch):
    """A bounded wait inside the tcgen05 kernel that expires (forced by a test switch: the first
    wait polls a barrier nothing arrives on) returns BCHDAV_ERR_TIMEOUT without faulting; the
    same handle then computes correctly."""
    import torch
    import paper_2212_04443_gb300 as P
    rng = synth.rng(5)
    n, k, nb = 20000, 64, 40
    V = rng.standard_normal((n, k)) / np.sqrt(n)
    Y = np.ascontiguousarray(np.linalg.qr(rng.standard_normal((k, k)))[0][:, :nb])
    Yd = torch.from_numpy(Y).cuda()
    monkeypatch.setenv("BCHDAV_TEST_EXPIRE_TC_WAIT", "1")
    with pytest.raises(P.BchdavError) as ei:
        H.rotate(torch.from_numpy(V.copy()).cuda(), Yd, nb, dense_path=0)
    assert ei.value.status == -6
    A = torch.from_numpy(V).cuda()
    with pytest.raises(P.BchdavError) as ei:
        H.gram(A, A[:, :7], dense_path=0)
    assert ei.value.status == -6
    monkeypatch.delenv("BCHDAV_TEST_EXPIRE_TC_WAIT")
    Vd = torch.from_numpy(V.copy()).cuda()
    H.rotate(Vd, Yd, nb, dense_path=0)
    assert np.abs(to_np(Vd)[:, :nb] - V @ Y).max() <= 1e-13 * np.abs(V @ Y).max()
    G = to_np(H.gram(A, A[:, :7].contiguous(), dense_path=0))
    assert np.abs(G - V.T @ V[:, :7]).max() <= 1e-13
