"""The allocation-free eigensolver entry point agrees with bchdav_eigh.

bchdav_eigh_noalloc serves callers that cannot allocate device memory when
they need the small eigensolver (another runtime owns the device memory pool,
or the path must not pay cudaMalloc's device-wide synchronisation); it works
in a fixed scratch array inside the library.  This file is collected last so
that a run stopping at the first failure has run every other test already.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _sym(n, seed):
    M = synth.rng(seed).standard_normal((n, n))
    return (M + M.T) / 2


def test_eigh_noalloc_matches_eigh_twice_in_a_row():
    import torch
    import paper_2212_04443_gb300 as P
    L = P.lib()
    handle = P.Handle()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, seed in ((96, 101), (128, 102)):   # two calls in a row on different matrices
        S = torch.from_numpy(_sym(n, seed)).cuda()
        D_ref, Y_ref = handle.eigh(S)
        D = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        Y = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        st = L.bchdav_eigh_noalloc(n, S.data_ptr(), n, D.data_ptr(), Y.data_ptr(), n, stream)
        assert st == 0, L.bchdav_last_error(None)
        D, Y, D_ref, Y_ref = (t.cpu().numpy() for t in (D, Y, D_ref, Y_ref))
        scale = max(1.0, np.abs(D_ref).max())
        assert np.abs(D - D_ref).max() <= 1e-13 * scale * n ** 0.5
        # same eigenvectors up to sign (columns of Y)
        sgn = np.sign(np.sum(Y * Y_ref, axis=0))
        assert np.abs(Y * sgn - Y_ref).max() <= 1e-10
        Sn = S.cpu().numpy()
        assert np.abs(Sn @ Y - Y * D).max() <= 1e-13 * scale * n


def test_eigh_noalloc_rejects_oversize():
    import torch
    import paper_2212_04443_gb300 as P
    L = P.lib()
    n = 129
    S = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    D = torch.zeros(n, dtype=torch.float64, device="cuda")
    Y = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    st = L.bchdav_eigh_noalloc(n, S.data_ptr(), n, D.data_ptr(), Y.data_ptr(), n, None)
    assert st == -1
    assert b"128" in L.bchdav_last_error(None)
