"""Write the oracle's results on the named workloads to tests/golden/*.json.

Calls only ``synth`` (inputs) and ``oracle`` (the float64 restatement of
Algorithm 2); nothing here touches the CUDA path.  Each file records the
sha256 of the edge list it was computed from, so a test can tell when the
generator produced a different graph on another host.

    python tests/golden/make_golden.py sbm10k sbm1m
    python tests/golden/make_golden.py --v0-cols k knn2m@200000 rmat24@18

``--v0-cols k`` starts from k Gaussian columns (V_init with k_init = k, taken b at a time by
Step 17) instead of b: on graphs whose zero eigenvalue has a multiplicity above b (one per
connected component) only such a start reaches the whole null space in exact arithmetic,
because the filter acts as the identity there (p(0) = 1).  Those files are named
``oracle_<workload>_v0k.json``.
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def edge_sha(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.src, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(g.dst, dtype=np.int32).tobytes())
    return h.hexdigest()


def main(names, v0_cols="b"):
    for name in names:
        w = synth.workload(name)
        g = w["graph"]
        L = oracle.laplacian_csr(g.n, g.src, g.dst)
        cols = w["k"] if v0_cols == "k" else w["b"]
        V0 = synth.gaussian_block(g.n, cols, w["v0_seed"])
        t0 = time.time()
        r = oracle.bchdav(L.scipy(), w["k"], w["b"], w["m"], w["act_max"], w["tol"], V_init=V0)
        dt = time.time() - t0
        res = oracle.relative_residuals(L.scipy(), r.evals, r.evecs)
        out = dict(
            workload=name, n=g.n, n_edges=int(g.n_edges), nnz=L.nnz, edge_sha256=edge_sha(g),
            k=w["k"], b=w["b"], m=w["m"], act_max=w["act_max"], tol=w["tol"], v0_seed=w["v0_seed"],
            v0_cols=cols,
            converged=bool(r.converged), iters=int(r.iters), n_spmm=int(r.n_spmm),
            evals=[float(x) for x in r.evals], max_rel_resid=float(res.max()),
            k_c_trajectory=[int(h["k_c"]) for h in r.history],
            k_act_trajectory=[int(h["k_act"]) for h in r.history],
            oracle_seconds=dt, host_cores=os.cpu_count(),
            produced_by="tests/golden/make_golden.py (oracle only)")
        suffix = "_v0k" if v0_cols == "k" else ""
        with open(os.path.join(HERE, f"oracle_{name}{suffix}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, cols, r.converged, r.iters, f"{dt:.1f}s", res.max())


if __name__ == "__main__":
    args = sys.argv[1:]
    mode = "b"
    if args[:1] == ["--v0-cols"]:
        mode = args[1]
        args = args[2:]
    main(args or ["sbm10k"], mode)
