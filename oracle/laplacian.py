"""Eq. (1): A = I - D^{-1/2} S D^{-1/2} of an undirected, unweighted graph (and, for general
bounds, the combinatorial Laplacian L = D - S of the same graph).

S_ij = 1 when i and j are joined by an edge (i != j), D_ii = sum_j S_ij.
Readings of what the paper leaves open:

* self loops are dropped and repeated edges count once (S is 0/1);
* a node of degree 0 gets A_ii = 1 and no off-diagonal entries (the pseudo
  inverse of D^{1/2} on that row), which keeps the spectrum inside [0, 2];
* canonical CSR: rows ascending, columns ascending within a row, the diagonal
  stored explicitly with value 1.0; off-diagonal value -(r_i * r_j) with
  r_i = 1.0 / sqrt(d_i), each operation IEEE correctly rounded;
* kind="combinatorial": L = D - S with the same pattern, diagonal d_i (0.0 for an isolated
  node), off-diagonal -1.0; spectrum in [0, 2 max_i d_i] (Gershgorin), the bounds of Sec. 2
  then come from Lanczos (oracle/lanczos.py).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int32 [n+1]
    colidx: np.ndarray  # int32 [nnz]
    val: np.ndarray     # float64 [nnz]
    degree: np.ndarray  # int64 [n], D_ii

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.colidx, self.rowptr), shape=(self.n, self.n))

    def dense(self) -> np.ndarray:
        return self.scipy().toarray()


def laplacian_csr(n: int, src, dst, kind: str = "normalized") -> CSR:
    """Symmetric normalized Laplacian (Eq. (1)) of the graph with the given edges, or with
    kind="combinatorial" the Laplacian D - S."""
    if kind not in ("normalized", "combinatorial"):
        raise ValueError(kind)
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("edge endpoint out of range")
    keep = src != dst
    u = np.concatenate([src[keep], dst[keep]])
    v = np.concatenate([dst[keep], src[keep]])
    keys = np.unique(u * n + v)              # S as sorted (row, col) pairs, once each
    rows = keys // n
    cols = keys % n
    deg = np.bincount(rows, minlength=n).astype(np.int64)   # D_ii = sum_j S_ij
    r = np.zeros(n, dtype=np.float64)
    has = deg > 0
    r[has] = 1.0 / np.sqrt(deg[has].astype(np.float64))      # D^{-1/2}
    if kind == "normalized":
        off = -(r[rows] * r[cols])                            # -(D^{-1/2} S D^{-1/2})_ij
        dval = np.ones(n)                                     # I on the diagonal
    else:
        off = -np.ones(rows.size)                             # -S_ij
        dval = deg.astype(np.float64)                         # D on the diagonal
    diag = np.arange(n, dtype=np.int64)
    all_rows = np.concatenate([rows, diag])
    all_cols = np.concatenate([cols, diag])
    all_val = np.concatenate([off, dval])
    order = np.argsort(all_rows * n + all_cols, kind="stable")
    colidx = all_cols[order].astype(np.int32)
    val = all_val[order]
    counts = np.bincount(all_rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, rowptr.astype(np.int32), colidx, val, deg)
