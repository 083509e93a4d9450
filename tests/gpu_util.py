"""Helpers shared by the GPU tests: build the Laplacian through the C-ABI and
compare against the oracle.  Only tests import this module."""
import numpy as np

import oracle
import synth


def device_csr(handle, g):
    """The library-built CSR of graph g (the product path of Eq. (1))."""
    import torch
    src = torch.from_numpy(np.ascontiguousarray(g.src, dtype=np.int32)).cuda()
    dst = torch.from_numpy(np.ascontiguousarray(g.dst, dtype=np.int32)).cuda()
    return handle.build_laplacian(g.n, src, dst)


def oracle_csr(g):
    return oracle.laplacian_csr(g.n, g.src, g.dst)


def to_np(t):
    return t.detach().cpu().numpy()


def residuals(A_scipy, evals, evecs):
    return oracle.relative_residuals(A_scipy, evals, evecs)


def null_space_basis(L):
    """Orthonormal basis of the null space of the Laplacian: D^{1/2} 1_C per component C."""
    import scipy.sparse.csgraph as csgraph
    ncomp, lab = csgraph.connected_components(L.scipy(), directed=False)
    sq = np.sqrt(L.degree.astype(float))
    iso = L.degree == 0
    U = np.zeros((L.n, ncomp))
    for c in range(ncomp):
        m = lab == c
        U[m, c] = sq[m]
    # isolated nodes have A_ii = 1: they contribute no null vector
    keep = np.linalg.norm(U, axis=0) > 0
    U = U[:, keep]
    U /= np.linalg.norm(U, axis=0)
    return U, int(keep.sum()), iso


def gaussian_v0(n, b, seed=0):
    import torch
    return torch.from_numpy(synth.gaussian_block(n, b, seed)).cuda()
