"""Algorithm 2: block Chebyshev-Davidson with inner-outer restart (Sec. 2).

Restated step by step in float64.  Readings of points the paper leaves open
(each is applied identically by the CUDA path):

* bounds: lowb = 0, upperb = 2 (normalized Laplacian, Sec. 2 and Sec. 4.1), or given (Lanczos);
  initial low_nwb = lowb + (upperb - lowb) * k_want / N.
* defaults: act_max = max(5 k_b, 30), dim_max = max(act_max + 2 k_b, k + 30)
  (Sec. 4), k_ri = max(floor(act_max/2), act_max - 3 k_b), k_ro = dim_max -
  2 k_b - k_c (Sec. 2, inner-outer restart).
* Step 5: the filter damps [low_nwb, upperb] and amplifies [lowb, low_nwb)
  (see ``filter``).
* Steps 9 and 12: Ritz values are taken in ascending order (the smallest
  eigenvalues are wanted; "non-increasing" in the listing is read as the order
  of the filtered operator's values).
* Step 11: the active block is V(:, k_c+1 : k_c+k_old) (the listing's
  k_c+1 : k_old is read as an offset typo).
* Step 12: the residual uses a fresh product A V(:, k_c+1 : k_c+k_b) (Sec. 3.4
  states that this step involves an SpMM); pair j is converged when
  ||A v_j - d_j v_j|| <= tol * ||v_j||.  Converged pairs among the k_b tested
  ones are moved to the front (stable partition of V, W and D) so that Steps
  14-15 apply to them.
* Step 13: returns the k_want smallest locked pairs in ascending order.
* Step 16: k_act = min(k_act, max(k_ro, k_b)), k_sub = k_c + k_act.
* Step 17: n_i = min(e_c, k_init - k_i) unused initial vectors, then the
  leading min(k_b - n_i, k_act) active Ritz vectors, then random vectors for
  any remainder.
* Step 18: low_nwb = median of the k_act non-converged Ritz values (mean of the
  middle two for an even count); kept unchanged when that median is not inside
  (lowb + 1e-12, upperb) or there is none.
* Step 2: k_i = min(k_b, k_init); missing columns are random vectors.
* the default dim_max is capped at N (a subspace cannot exceed the problem).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .dgks import dgks_orthonormalize, TAU_DEP_F64
from .filter import chebyshev_filter
from .philox import uniform_pm_half, STREAM_FILL

LOWB = 0.0
UPPERB = 2.0
LOW_NWB_EPS = 1e-12


def default_params(n: int, k: int, b: int, act_max: int | None = None, dim_max: int | None = None):
    """Paper defaults (Sec. 4); dim_max is capped at N so tiny problems stay well posed."""
    act = act_max if act_max else max(5 * b, 30)
    dmax = dim_max if dim_max else min(max(act + 2 * b, k + 30), n)
    k_ri = max(act // 2, act - 3 * b)
    return act, dmax, k_ri


@dataclass
class BchdavResult:
    evals: np.ndarray
    evecs: np.ndarray
    converged: bool
    iters: int
    n_spmm: int
    history: list = field(default_factory=list)


def _median(x: np.ndarray) -> float:
    s = np.sort(x)
    n = s.shape[0]
    if n % 2 == 1:
        return float(s[n // 2])
    return 0.5 * (float(s[n // 2 - 1]) + float(s[n // 2]))


def relative_residuals(A, evals, evecs) -> np.ndarray:
    """||A v - lambda v||_2 / ||v||_2 per column, with a fresh product A V."""
    R = A @ evecs - evecs * evals[None, :]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(evecs, axis=0)


def bchdav(A, k_want: int, b: int, m: int, act_max: int | None, tol: float, *,
           V_init: np.ndarray | None = None, dim_max: int | None = None, itmax: int = 1000,
           seed: int = 0, tau_dep: float = TAU_DEP_F64, record: bool = True,
           max_iters_run: int | None = None, bounds: tuple | None = None) -> BchdavResult:
    """k_want smallest eigenpairs of the symmetric operator A with spectrum in [0, 2], or in
    [lowb, upperb] given as ``bounds`` (e.g. from oracle/lanczos.py for matrices whose bounds
    are not analytic, Sec. 2).

    ``A`` is a scipy sparse matrix (or anything with ``@`` and ``shape``).
    ``max_iters_run`` stops early (for bounded timing samples) without error.
    """
    N = A.shape[0]
    if not (1 <= k_want <= N and b >= 1 and m >= 1):
        raise ValueError("bad sizes")
    act_max, dim_max, k_ri = default_params(N, k_want, b, act_max, dim_max)
    if act_max < 2 * b or act_max > N:
        raise ValueError("act_max must satisfy 2 k_b <= act_max <= N")
    ncols = max(dim_max, k_want + 2 * b)
    if ncols > N:
        raise ValueError("subspace larger than the problem")

    # Step 1: bounds.
    lowb, upperb = (LOWB, UPPERB) if bounds is None else (float(bounds[0]), float(bounds[1]))
    if not upperb > lowb:
        raise ValueError("bounds: need lowb < upperb")
    low_nwb = lowb + (upperb - lowb) * k_want / N

    # Step 2: first filter input.
    k_init = 0 if V_init is None else V_init.shape[1]
    n_first = min(b, k_init)
    V_tmp = np.empty((N, b))
    if n_first:
        V_tmp[:, :n_first] = V_init[:, :n_first]
    fill_counter = 0
    for j in range(n_first, b):
        V_tmp[:, j] = uniform_pm_half(N, fill_counter, STREAM_FILL, seed)
        fill_counter += 1
    k_i = n_first

    # Step 3: counters.
    k_c = 0
    k_sub = 0
    k_act = 0
    V = np.zeros((N, ncols))
    W = np.zeros((N, act_max))
    H = np.zeros((act_max, act_max))
    eval_locked: list[float] = []
    rep_counter = 0
    n_spmm = 0
    history = []

    it = 0
    while it < itmax:
        if max_iters_run is not None and it >= max_iters_run:
            break
        it += 1
        # Step 5: Chebyshev filter (Algorithm 3) of V_tmp.
        Xf = chebyshev_filter(A, V_tmp, m, low_nwb, upperb, lowb)
        n_spmm += m
        # Step 6: orthonormalise against V(:, 1:k_sub).
        Q, n_rep, rep_counter = dgks_orthonormalize(V[:, :k_sub], Xf, seed=seed,
                                                    rep_counter=rep_counter, tau_dep=tau_dep)
        V[:, k_sub:k_sub + b] = Q
        # Step 7: W(:, k_act+1:k_act+b) = A V_new.
        W[:, k_act:k_act + b] = A @ Q
        n_spmm += 1
        k_act += b
        k_sub += b
        # Step 8: last k_b columns of H, then symmetrise.
        Hnew = V[:, k_c:k_sub].T @ W[:, k_act - b:k_act]
        H[:k_act, k_act - b:k_act] = Hnew
        H[k_act - b:k_act, :k_act - b] = Hnew[:k_act - b, :].T
        blk = H[k_act - b:k_act, k_act - b:k_act]
        H[k_act - b:k_act, k_act - b:k_act] = 0.5 * (blk + blk.T)
        # Step 9: H Y = Y D, ascending.
        D, Y = np.linalg.eigh(H[:k_act, :k_act])
        k_old = k_act
        # Step 10: inner restart.
        if k_act + b > act_max:
            k_act = k_ri
            k_sub = k_act + k_c
        # Step 11: subspace rotation.
        V[:, k_c:k_c + k_act] = V[:, k_c:k_c + k_old] @ Y[:k_old, :k_act]
        W[:, :k_act] = W[:, :k_old] @ Y[:k_old, :k_act]
        D = D[:k_act].copy()
        # Step 12: residuals of the k_b leading Ritz pairs, convergence, locking.
        nt = min(b, k_act)
        Vt = V[:, k_c:k_c + nt]
        R = A @ Vt - Vt * D[None, :nt]
        n_spmm += 1
        rn = np.linalg.norm(R, axis=0)
        vn = np.linalg.norm(Vt, axis=0)
        conv = rn <= tol * vn
        order = np.concatenate([np.flatnonzero(conv), np.flatnonzero(~conv)])
        V[:, k_c:k_c + nt] = V[:, k_c + order]
        W[:, :nt] = W[:, order]
        D[:nt] = D[order]
        e_c = int(conv.sum())
        eval_locked.extend(D[:e_c].tolist())
        k_c += e_c
        if record:
            history.append(dict(it=it, k_c=k_c, e_c=e_c, k_act=k_act, k_sub=k_sub, k_old=k_old,
                                low_nwb=low_nwb, resid=(rn / vn).tolist(), n_rep=n_rep,
                                ritz=D[:nt].tolist()))
        # Step 13: exit.
        if k_c >= k_want:
            ev = np.array(eval_locked)
            idx = np.argsort(ev, kind="stable")[:k_want]
            return BchdavResult(ev[idx], V[:, idx].copy(), True, it, n_spmm, history)
        # Step 14: drop converged columns of W.
        if e_c > 0:
            W[:, :k_act - e_c] = W[:, e_c:k_act].copy()
            k_act -= e_c
        # Step 15: H = diag of the non-converged Ritz values.
        d_act = D[e_c:e_c + k_act].copy()
        H[:, :] = 0.0
        H[np.arange(k_act), np.arange(k_act)] = d_act
        # Step 16: outer restart.
        if k_sub + b > dim_max:
            k_ro = dim_max - 2 * b - k_c
            k_act = min(k_act, max(k_ro, b))
            k_sub = k_c + k_act
        # Step 17: next filter input.
        n_i = min(e_c, k_init - k_i) if k_init > k_i else 0
        n_r = min(b - n_i, k_act)
        n_x = b - n_i - n_r
        if n_i:
            V_tmp[:, :n_i] = V_init[:, k_i:k_i + n_i]
        V_tmp[:, n_i:n_i + n_r] = V[:, k_c:k_c + n_r]
        for j in range(n_x):
            V_tmp[:, n_i + n_r + j] = uniform_pm_half(N, fill_counter, STREAM_FILL, seed)
            fill_counter += 1
        k_i += n_i
        # Step 18: new cut from the median of the non-converged Ritz values.
        if k_act > 0:
            med = _median(d_act[:k_act])
            if lowb + LOW_NWB_EPS < med < upperb:
                low_nwb = med
    ev = np.array(eval_locked)
    idx = np.argsort(ev, kind="stable")
    return BchdavResult(ev[idx], V[:, idx].copy(), False, it, n_spmm, history)
