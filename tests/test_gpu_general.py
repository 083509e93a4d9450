"""General symmetric matrices on the GPU (Sec. 2: bounds from standard Lanczos when they are not
analytic): the combinatorial Laplacian D - S built bit-exactly, the k-step Lanczos estimate
(bchdav_lanczos_bounds) against oracle/lanczos.py, and Algorithm 2 with estimated or given bounds
on the combinatorial Laplacian and on an indefinite sparse matrix, against dense brute force and
the oracle's solve with the oracle's bounds."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_np
from oracle import lanczos as LZ

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import paper_2212_04443_gb300 as P
    return P.Handle()


def _comb_device(H, g):
    import torch
    import paper_2212_04443_gb300 as P
    return H.build_laplacian(g.n, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda(),
                             kind=P.LAPLACIAN_COMBINATORIAL)


def _device_csr(M):
    """A caller-built CSR (both triangles stored) in torch CUDA tensors."""
    import torch
    import paper_2212_04443_gb300 as P
    M = M.tocsr()
    M.sort_indices()
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    return P.DeviceCSR(M.shape[0], t(M.indptr, np.int32), t(M.indices, np.int32),
                       t(M.data, np.float64), t(M.data.astype(np.float32), np.float32))


GRAPHS = {
    "sbm": lambda: synth.sbm_edges(20011, 8, d_in=12, d_out=2, seed=21),
    # a hub longer than the SpMM segment length, power-law rows and isolated nodes
    "hub": lambda: synth.disjoint_union(synth.star_edges(2100), synth.rmat_edges(11, seed=22),
                                        synth.path_edges(1), synth.path_edges(1)),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_combinatorial_laplacian_bit_exact(H, name):
    g = GRAPHS[name]()
    A = _comb_device(H, g)
    L = oracle.laplacian_csr(g.n, g.src, g.dst, kind="combinatorial")
    assert np.array_equal(to_np(A.rowptr), L.rowptr)
    assert np.array_equal(to_np(A.colidx), L.colidx)
    assert np.array_equal(to_np(A.val), L.val)
    assert np.array_equal(to_np(A.val_f32), L.val.astype(np.float32))


def _indefinite(n=3000, seed=23):
    """Sparse symmetric matrix with eigenvalues of both signs: a random sparse pattern with
    normal values plus a normal diagonal."""
    import scipy.sparse as sp
    g = synth.rng(seed)
    m = 6 * n
    i, j = g.integers(0, n, m), g.integers(0, n, m)
    S = sp.coo_matrix((g.standard_normal(m), (i, j)), shape=(n, n)).tocsr()
    S = S + S.T + sp.diags(g.standard_normal(n) * 2.0)
    S.sum_duplicates()
    return S.tocsr()


@pytest.mark.parametrize("case,steps", [("comb", 10), ("comb", 20), ("norm", 20), ("hub", 32),
                                        ("indef", 20), ("indef", 64)])
def test_lanczos_matches_oracle(H, case, steps):
    import torch
    if case == "indef":
        M = _indefinite()
        A = _device_csr(M)
    else:
        g = GRAPHS["hub" if case == "hub" else "sbm"]()
        kind = "normalized" if case == "norm" else "combinatorial"
        L = oracle.laplacian_csr(g.n, g.src, g.dst, kind=kind)
        M = L.scipy()
        if kind == "normalized":
            A = H.build_laplacian(g.n, torch.from_numpy(g.src).cuda(),
                                  torch.from_numpy(g.dst).cuda())
        else:
            A = _comb_device(H, g)
    import scipy.sparse.linalg as sla
    lo, hi, alpha, beta = H.lanczos_bounds(A, steps, seed=5)
    lo_o, hi_o, alpha_o, beta_o = LZ.bounds(M, steps, 5)
    scale = abs(hi_o) + abs(lo_o)
    assert alpha.size == alpha_o.size == steps
    # Without reorthogonalisation, two runs in floating point part ways once a Ritz value has
    # converged and the basis loses orthogonality; the coefficients are compared element by
    # element while the oracle's basis is orthonormal to 1e-9, the bounds always by what any
    # run guarantees (the upper bound above the largest eigenvalue, the lower one a Ritz value).
    _, _, Vo = LZ.lanczos(M, LZ.start_vector(M.shape[0], 5), steps)
    p = 0
    while p < steps and np.abs(Vo[:, :p + 1].T @ Vo[:, :p + 1] - np.eye(p + 1)).max() <= 1e-9:
        p += 1
    assert p >= min(steps, 8)
    assert np.allclose(alpha[:p], alpha_o[:p], rtol=0, atol=1e-10 * scale)
    assert np.allclose(beta[:p], beta_o[:p], rtol=0, atol=1e-10 * scale)
    if p == steps:
        assert abs(lo - lo_o) <= 1e-10 * scale and abs(hi - hi_o) <= 1e-10 * scale
    lmax = sla.eigsh(M, k=1, which="LA", return_eigenvectors=False, tol=1e-12)[0]
    lmin = sla.eigsh(M, k=1, which="SA", return_eigenvectors=False, tol=1e-12, maxiter=100000)[0]
    assert hi >= lmax - 1e-9 * scale
    assert lmin - 1e-9 * scale <= lo <= lmax + 1e-9 * scale


def test_lanczos_argument_errors(H):
    import paper_2212_04443_gb300 as P
    A = _comb_device(H, synth.cycle_edges(30))
    for steps in (0, 65, 31):
        with pytest.raises(P.BchdavError):
            H.lanczos_bounds(A, steps)


@pytest.mark.parametrize("precision", [0, 1])
def test_combinatorial_solve_with_lanczos_bounds(H, precision):
    g = synth.sbm_edges(3000, 6, d_in=10, d_out=1.5, seed=24)
    A = _comb_device(H, g)
    L = oracle.laplacian_csr(g.n, g.src, g.dst, kind="combinatorial")
    k, b, m, act, tol = 6, 6, 11, 36, 1e-8
    ev, V, info = H.solve(A, k, b, m, act, tol, precision=precision, bounds="lanczos")
    assert info.status == 0
    lo_o, hi_o, _, _ = LZ.bounds(L.scipy(), 20, 0)
    assert abs(info.lowb - lo_o) <= 1e-10 * hi_o and abs(info.upperb - hi_o) <= 1e-10 * hi_o
    w = np.linalg.eigvalsh(L.dense())
    ev, V = to_np(ev), to_np(V)
    assert np.allclose(ev, w[:k], atol=1e-8 * hi_o)
    assert oracle.relative_residuals(L.scipy(), ev, V).max() <= tol * 1.0001
    r = oracle.bchdav(L.scipy(), k, b, m, act, tol, bounds=(lo_o, hi_o))
    assert r.converged and np.allclose(ev, r.evals, atol=1e-9 * hi_o)


@pytest.mark.parametrize("mode", ["lanczos", "given"])
@pytest.mark.parametrize("precision", [0, 1])
def test_indefinite_solve(H, mode, precision):
    M = _indefinite()
    A = _device_csr(M)
    Md = M.toarray()
    w = np.linalg.eigvalsh(Md)
    if mode == "given":   # Gershgorin discs
        rad = np.abs(Md).sum(axis=1) - np.abs(np.diag(Md))
        bounds = (float((np.diag(Md) - rad).min()), float((np.diag(Md) + rad).max()))
    else:
        bounds = "lanczos"
    k, b, m, act, tol = 8, 8, 13, 48, 1e-8
    ev, V, info = H.solve(A, k, b, m, act, tol, precision=precision, bounds=bounds,
                          lanczos_steps=30)
    assert info.status == 0, info
    assert w[0] < 0 < w[-1]
    ev, V = to_np(ev), to_np(V)
    assert np.allclose(ev, w[:k], atol=1e-8 * np.abs(w).max())
    assert oracle.relative_residuals(M, ev, V).max() <= tol * 1.0001


def test_bounds_option_errors(H):
    import paper_2212_04443_gb300 as P
    A = _comb_device(H, synth.sbm_edges(500, 2, d_in=8, d_out=1, seed=25))
    with pytest.raises(P.BchdavError):
        H.solve(A, 2, 2, 5, 10, 1e-8, bounds=(1.0, 1.0))
    with pytest.raises(P.BchdavError):
        H.solve(A, 2, 2, 5, 10, 1e-8, bounds="lanczos", lanczos_steps=65)
