"""Host-side logic of the binding and the bench that needs no GPU: the Step 1 bounds options
marshalled into bchdav_opts, and the oracle problem the bench builds for a workload (matrix
kind and Lanczos bounds)."""
import os
import sys

import numpy as np
import pytest

import oracle
import synth
from oracle import lanczos

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_options_marshalling():
    import paper_2212_04443_gb300 as P
    o = P.OptsStruct()
    P._set_bounds(o, None, 0)
    assert o.bounds == P.BOUNDS_NORMALIZED
    P._set_bounds(o, (-1.5, 7.25), 0)
    assert o.bounds == P.BOUNDS_GIVEN and (o.lowb, o.upperb) == (-1.5, 7.25)
    P._set_bounds(o, "lanczos", 30)
    assert o.bounds == P.BOUNDS_LANCZOS and o.lanczos_steps == 30
    with pytest.raises(ValueError):
        P._set_bounds(o, "gershgorin", 0)


def test_bench_oracle_problem_for_the_combinatorial_workload():
    sys.path.insert(0, ROOT)
    from bench import oracle_problem
    w = synth.workload("sbm1m_comb@3000")
    A, bnd = oracle_problem(w)
    g = w["graph"]
    L = oracle.laplacian_csr(g.n, g.src, g.dst, kind="combinatorial")
    assert (A != L.scipy()).nnz == 0
    lo, hi, _, _ = lanczos.bounds(L.scipy(), 20, 0)
    assert bnd == (lo, hi)
    A0, b0 = oracle_problem(synth.workload("sbm10k"))
    assert b0 is None and np.allclose(A0.diagonal()[np.diff(A0.indptr) > 0], 1.0)
