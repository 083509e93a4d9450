"""Plain FP64 CPU oracle of the block Chebyshev-Davidson eigensolver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, calls or
links this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with the CUDA path: both consume the same seeded inputs from
``synth`` and nothing else.

The oracle restates the paper's method step by step in float64 numpy, with
library primitives (scipy CSR times dense block, numpy matmul, LAPACK eigh,
sort) standing in for single steps and no blocking or fusion beyond what the
paper states:

* ``laplacian``  the symmetric normalized Laplacian of Eq. (1) as CSR;
* ``filter``     the scaled Chebyshev filter of Algorithm 3 and the closed
                 form of the polynomial it applies (Eqs. (3)-(5));
* ``dgks``       orthonormalisation of a new block against the basis with
                 DGKS re-orthogonalisation and random replacement (Sec. 2);
* ``bchdav``     Algorithm 2, block Chebyshev-Davidson with inner-outer restart
                 and progressive filtering;
* ``philox``     the Philox4x32-10 counter-based generator (Salmon et al.,
                 SC 2011) that draws replacement vectors inside the method;
* ``gnn``        the learned start block (an extension feeding V_init): network,
                 subspace-alignment loss, its gradient, Adam, Ritz ordering;
* ``cluster``    Algorithm 1, Steps 4-5: row normalisation of the eigenvectors and
                 Lloyd's k-means on the rows; adjusted Rand index and NMI;
* ``lanczos``    spectrum bounds by k-step Lanczos for matrices without analytic bounds
                 (Sec. 2), e.g. the combinatorial Laplacian D - S (``laplacian``, kind).

Pins (tests/test_oracle_*.py, run with ``-m "not gpu"``): closed-form spectra
of cycles, paths, hypercubes, complete and complete-bipartite graphs and their
disjoint unions; the closed-form filter polynomial on exact eigenvectors; dense
brute-force eigendecomposition for N <= 200; invariants (spectrum in [0, 2],
lambda_1 = 0 with eigenvector D^{1/2} 1, zero multiplicity = number of
connected components); hand-computed Laplacian entries; published Philox
known-answer vectors.  Iteration counts and timings have no printed value in
the paper: parity unpinned for those (compared GPU-vs-oracle only).
"""
from .laplacian import laplacian_csr, CSR  # noqa: F401
from .filter import chebyshev_filter, filter_polynomial, chebyshev_T  # noqa: F401
from .philox import philox4x32_10, uniform_pm_half  # noqa: F401
from .dgks import dgks_orthonormalize  # noqa: F401
from .bchdav import bchdav, BchdavResult, default_params, relative_residuals  # noqa: F401
from . import gnn  # noqa: F401
from . import cluster  # noqa: F401
from . import lanczos  # noqa: F401
