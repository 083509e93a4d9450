"""Parity with the oracle at the configured workloads, through the C-ABI.

* The 1,000,000-node SBM that bench.py times (100 clusters, k = 100, b = 20, m = 15,
  act_max = 300): the library-built CSR bit for bit against the oracle's; the float64 path's
  eigenvalues within 1e-10 of the oracle's (tests/golden/oracle_sbm1m.json, same iteration
  count and k_c trajectory); the mixed path's eigenvalue error against the same golden (reported,
  and bounded by the residual tolerance: 4 tol^2 / gap per eigenvalue), every residual
  recomputed by scipy, orthonormality and lambda_1 = 0 with eigenvector D^{1/2} 1.
* The kNN-GMM workload reduced to 200,000 points (50 mixture components, 10-NN; k = 50,
  b = 10, m = 13, act_max = 150) and R-MAT at scale 18 (k = 64, b = 16, m = 15,
  act_max = 192), both with zero eigenvalues of multiplicity (= connected components) above
  b: started, like their goldens, from k Gaussian columns (their null-space components span
  the whole null space, which the filter leaves unchanged, p(0) = 1, while a b-column start
  reaches more of it only through rounding noise).  Checked: eigenvalues within 1e-10 of the
  oracle's, the same count of zero eigenvalues (50 of 50 components on the kNN graph), the
  null vectors inside span{D^{1/2} 1_C} (closed form), residuals, orthonormality.
  Inside the null space any orthonormal basis is correct and which Ritz vectors are tested
  first is decided by rounding.  On the kNN graph both paths still follow the oracle's lock
  counts at every iteration (asserted for float64).  On R-MAT the trajectories part after
  about 11 iterations and the number of null directions locked before k pairs are reached
  depends on rounding (the oracle: 42 of 49); there the float64 path happens to return the
  oracle's eigenvalues, and for both paths the positive eigenvalues are compared on their
  common prefix (the smallest ones, unique) and the null vectors by membership.
"""
import hashlib
import json
import os

import numpy as np
import pytest
import scipy.sparse.csgraph as csgraph

import synth
from gpu_util import device_csr, null_space_basis, oracle_csr, residuals, to_np

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def edge_sha(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.src, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(g.dst, dtype=np.int32).tobytes())
    return h.hexdigest()


def v0_of(n, cols, seed):
    import torch
    return torch.from_numpy(synth.gaussian_block(n, cols, seed)).cuda()


@pytest.fixture(scope="module")
def H():
    import paper_2212_04443_gb300 as P
    return P.Handle()


@pytest.fixture(scope="module")
def sbm1m(H):
    w = synth.workload("sbm1m")
    g = w["graph"]
    gold = load_golden("oracle_sbm1m.json")
    assert edge_sha(g) == gold["edge_sha256"], "the generator produced another graph"
    L = oracle_csr(g)
    A = device_csr(H, g)
    return w, g, gold, L, A


def test_sbm1m_csr_bit_exact(H, sbm1m):
    """Eq. (1) at the bench's size: the library's CSR (multi-tile scan, sort and fill stages)
    equals the oracle's bit for bit, float32 copy included."""
    w, g, gold, L, A = sbm1m
    assert A.n == L.n == 1_000_000 and A.nnz == L.nnz == gold["nnz"]
    assert np.array_equal(to_np(A.rowptr), L.rowptr)
    assert np.array_equal(to_np(A.colidx), L.colidx)
    assert np.array_equal(to_np(A.val).view(np.uint64), L.val.view(np.uint64))
    assert np.array_equal(to_np(A.val_f32), L.val.astype(np.float32))
    assert H.check_csr(A) == 0


def test_sbm1m_fp64_matches_oracle_golden(H, sbm1m):
    import paper_2212_04443_gb300 as P
    w, g, gold, L, A = sbm1m
    k, b, m, act, tol = w["k"], w["b"], w["m"], w["act_max"], w["tol"]
    V0 = v0_of(g.n, b, w["v0_seed"])
    ev, V, info = H.solve(A, k, b, m, act, tol, v_init=V0, precision=P.PREC_FP64, itmax=200,
                          record_history=True)
    hist = H.history()
    assert info.status == 0
    ev = to_np(ev)
    err = np.abs(ev - np.asarray(gold["evals"])).max()
    print(f"sbm1m float64 path: max |lambda - lambda_oracle| = {err:.3e}, iters {info.iters}")
    assert err <= 1e-10
    assert info.iters == gold["iters"]
    assert [h.k_c for h in hist] == gold["k_c_trajectory"]
    assert residuals(L.scipy(), ev, to_np(V)).max() <= tol * 1.0001


def test_sbm1m_mixed_properties_and_error(H, sbm1m):
    """The bench's own configuration (mixed precision, slice products)."""
    import paper_2212_04443_gb300 as P
    w, g, gold, L, A = sbm1m
    k, b, m, act, tol = w["k"], w["b"], w["m"], w["act_max"], w["tol"]
    V0 = v0_of(g.n, b, w["v0_seed"])
    ev, V, info = H.solve(A, k, b, m, act, tol, v_init=V0, precision=P.PREC_MIXED, itmax=200,
                          record_history=True)
    hist = H.history()
    assert info.status == 0
    ev, V = to_np(ev), to_np(V)
    As = L.scipy()
    assert csgraph.connected_components(As, directed=False)[0] == 1
    assert residuals(As, ev, V).max() <= tol * 1.0001
    assert np.abs(V.T @ V - np.eye(k)).max() < 1e-10
    assert np.all(np.diff(ev) >= -1e-14) and ev[0] > -1e-10 and ev[-1] < 2
    assert abs(ev[0]) < 1e-10
    u = np.sqrt(L.degree.astype(float))
    u /= np.linalg.norm(u)
    assert abs(abs(u @ V[:, 0]) - 1.0) < 1e-10
    gev = np.asarray(gold["evals"])
    dev = np.abs(ev - gev)
    err = dev.max()
    print(f"sbm1m mixed path: max |lambda - lambda_oracle| = {err:.3e}, iters {info.iters} "
          f"(oracle {gold['iters']}), k_c {[h.k_c for h in hist]}")
    # The mixed path follows another trajectory (float32 filter, truncated products), so its
    # converged vectors differ from the oracle's within the residual tolerance.  A Ritz value
    # with residual r is within r^2 / gap of its eigenvalue (gap: distance to the rest of the
    # spectrum), so the two runs' eigenvalues may differ by up to 2 tol^2 / gap: 3.2e-10 at
    # this spectrum's smallest gap, 6.2e-7.  Gaps from the oracle's eigenvalues (the last one's
    # left gap only), with a factor 2 for the gap estimate.
    gaps = np.minimum(np.r_[np.inf, np.diff(gev)], np.r_[np.diff(gev), np.inf])
    bound = 4 * tol ** 2 / gaps + 1e-12
    assert np.all(dev <= bound), (dev / bound).max()


def _degenerate_case(H, name, precision, orth_tol=None, exact_set=True):
    import paper_2212_04443_gb300 as P
    w = synth.workload(name)
    g = w["graph"]
    gold = load_golden(f"oracle_{name}_v0k.json")
    assert edge_sha(g) == gold["edge_sha256"], "the generator produced another graph"
    k, b, m, act, tol = w["k"], w["b"], w["m"], w["act_max"], w["tol"]
    assert gold["v0_cols"] == k
    L = oracle_csr(g)
    A = device_csr(H, g)
    ev, V, info = H.solve(A, k, b, m, act, tol, v_init=v0_of(g.n, k, w["v0_seed"]),
                          precision=precision, itmax=400, record_history=True)
    hist = H.history()
    assert info.status == 0
    ev, V = to_np(ev), to_np(V)
    res = residuals(L.scipy(), ev, V).max()
    ortho = np.abs(V.T @ V - np.eye(k)).max()
    gev = np.asarray(gold["evals"])
    err = np.abs(ev - gev).max()
    U, ncomp, _ = null_space_basis(L)
    zero = np.abs(ev) < 1e-10
    Z = V[:, zero]
    dist = np.linalg.norm(Z - U @ (U.T @ Z), axis=0).max()
    gk = gold["k_c_trajectory"]
    got = [h.k_c for h in hist]
    same = 0
    for a, o in zip(got, gk):
        if a != o:
            break
        same += 1
    print(f"{name} {'float64' if precision == 0 else 'mixed'}: {ncomp} components, "
          f"{int(zero.sum())} zero eigenvalues (oracle {int(np.sum(np.abs(gev) < 1e-10))}), "
          f"max |lambda - lambda_oracle| = {err:.3e}, max residual {res:.2e}, "
          f"|V^T V - I| {ortho:.2e}, null-space distance {dist:.2e}, iters {info.iters} "
          f"(oracle {gold['iters']}), k_c agree for the first {same} iterations; gpu {got} "
          f"oracle {gk}")
    assert res <= tol * 1.0001
    # the slice products' error bound grows with the largest entry of each 1024-row chunk:
    # power-law graphs (hub rows) end near 1e-12 on the float64 path; the mixed path's
    # 36-bit rotation operands add about 2e-11 per rotation over the iterations
    assert ortho < (orth_tol if orth_tol else (1e-12 if precision == P.PREC_FP64 else 1e-10))
    # null vectors lie in span{D^{1/2} 1_C}, within residual / gap (the gap at least the
    # smallest positive eigenvalue returned), at most one per component
    pos = ev[~zero]
    gap = pos.min() if pos.size else 1.0
    assert int(zero.sum()) <= ncomp
    assert dist <= 4 * tol / gap
    if exact_set:
        assert int(zero.sum()) == int(np.sum(np.abs(gev) < 1e-10))
        assert err <= 1e-10
    else:
        # Step 17 hands out the start columns only as pairs lock, so the iteration can reach
        # k locked pairs while start columns carrying null directions are still unused (on
        # R-MAT the oracle returns 42 of the 49 zero eigenvalues and 22 positive ones); how
        # many null directions are locked by then depends on rounding.  What is unique: the
        # positive eigenvalues returned are the smallest ones, so both runs' positive
        # eigenvalues agree on their common prefix.
        gpos = gev[np.abs(gev) >= 1e-10]
        c = min(pos.size, gpos.size)
        assert c >= 1 and np.abs(pos[:c] - gpos[:c]).max() <= 1e-10
    return info, got, gk, same


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_knn200k_matches_oracle_golden(H, precision):
    info, got, gk, same = _degenerate_case(H, "knn2m@200000", precision)
    if precision == 0:
        assert same == len(gk) == len(got)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_rmat18_matches_oracle_golden(H, precision):
    info, got, gk, same = _degenerate_case(H, "rmat24@18", precision,
                                           orth_tol=5e-12 if precision == 0 else 1e-9,
                                           exact_set=False)
    assert info.iters <= 2 * len(gk)
