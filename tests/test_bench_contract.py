"""bench.py on the CPU: the reference arm's JSON line carries the contract's keys, and the
partition scores the clustering leg reports agree with the oracle's (pinned against
scikit-learn and hand-computed values)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from oracle import cluster

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_line_keys():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "sbm10k", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["higher_is_better"] is False
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1


def test_bench_scores_match_the_oracle():
    sys.path.insert(0, ROOT)
    from bench import partition_scores
    g = synth.rng(3)
    for _ in range(4):
        a = g.integers(0, 7, 3000)
        b = np.where(g.random(3000) < 0.7, a, g.integers(0, 5, 3000))
        ari, nmi = partition_scores(a, b)
        assert ari == pytest.approx(cluster.adjusted_rand_index(a, b), abs=1e-12)
        assert nmi == pytest.approx(cluster.normalized_mutual_info(a, b), abs=1e-12)
    assert partition_scores([0, 0, 1, 1], [0, 0, 1, 2])[0] == pytest.approx(4 / 7)


def test_filter_model_bytes_follow_the_scope_table():
    """Compulsory filter bytes: per step 4 (N + 1) + nnz (4 + s) + 3 N b s, the first step of a
    filter 2 N b s; the 1M-node SBM (nnz 18,988,714, b = 20, float32) moves 395.9 MB per full
    step and 315.9 MB in its first."""
    sys.path.insert(0, ROOT)
    from bench import filter_model_bytes
    n, nnz, b = 1_000_000, 18_988_714, 20
    one = filter_model_bytes(n, nnz, b, 1, 1, 4.0)
    two = filter_model_bytes(n, nnz, b, 2, 1, 4.0)
    assert one == pytest.approx(4 * (n + 1) + nnz * 8 + 2 * n * b * 4)
    assert two - one == pytest.approx(4 * (n + 1) + nnz * 8 + 3 * n * b * 4)
    assert round((two - one) / 1e6, 1) == 395.9 and round(one / 1e6, 1) == 315.9
    assert filter_model_bytes(n, nnz, b, 15, 16, 4.0) == pytest.approx(16 * (one + 14 * (two - one)))


def test_slice_pair_work_follows_the_precision_schedule():
    """The tensor-core work the bench charges per component: 36 pairs (8 slices) on the float64
    path; on the mixed path 10 pairs (4 slices) for the first DGKS Gram product, 21 for Step 11
    and 36 for Step 8."""
    sys.path.insert(0, ROOT)
    from types import SimpleNamespace as NS
    from bench import h_flops, orth_flops, pair_work, rotation_flops
    n, b = 1000, 4
    hist = [NS(k_orth=8, k_old=12, k_act=16, min_resid=r) for r in (1e-1, 1e-3, 5e-5, 1e-9)]
    for name, f in (("rotation", rotation_flops(hist, n)),
                    ("orthonormalisation", orth_flops(hist, n, b)),
                    ("rayleigh_quotient", h_flops(hist, n, b))):
        assert pair_work(name, hist, n, b, False) == 36 * f
    assert pair_work("rotation", hist, n, b, True) == 21 * rotation_flops(hist, n)
    assert pair_work("rayleigh_quotient", hist, n, b, True) == 36 * h_flops(hist, n, b)
    dg = 2.0 * n * 8 * b
    rest = 6.0 * n * 8 * b + 4.0 * n * b * b
    assert pair_work("orthonormalisation", hist, n, b, True) == 4 * (10 * dg + 36 * rest)
