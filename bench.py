#!/usr/bin/env python
"""Time to k eigenpairs at relative residual 1e-8 on one GB300, plus the filter
SpMM's HBM bandwidth against the measured peak.

Workload (one "step" = one full block Chebyshev-Davidson solve, Algorithm 2,
of every step from the filter to the final residual check): stochastic block
model, N = 1,000,000 nodes, 100 equal clusters, expected intra-degree 16,
inter-degree 2, normalized Laplacian (Eq. (1)) built on the device; k = 100,
k_b = 20, m = 15, act_max = 300, tol = 1e-8, Gaussian V0 (seed 0).  The
headline path is the mixed one (float32 filter recurrence, float64 elsewhere);
the float64 path is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs independent replicas (the method has no data-parallel exchange on
one problem); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "time to k eigenpairs at rel. residual 1e-8; filter SpMM HBM GB/s vs peak"
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 float64 rate (2 DFMA/clk/SM x 152 SMs x 2.07 GHz)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sbm1m")
    ap.add_argument("--workers", type=int, default=8, help="concurrent solves of a batch workload")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched leg (the batch512 workload: 512 SBM graphs)")
    ap.add_argument("--batch-graphs", type=int, default=512,
                    help="graphs of the batch512 workload the batched leg solves (its first ones)")
    ap.add_argument("--no-warm-start", action="store_true",
                    help="skip the learned start-block leg (a network trained on three graphs of "
                         "the workload's family, evaluated on a held-out one)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cluster", action="store_true",
                    help="skip Steps 4-5 (row normalisation + k-means) after the solve")
    ap.add_argument("--dense-path", type=int, default=0, choices=[0, 1, 2],
                    help="0: slice products on tcgen05 (default); 1: float64 FMA kernels; "
                         "2: slice products on the legacy warp-level mma")
    return ap.parse_args()


def load_bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        # the products run inside a long solve: the sustained figure
        return float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured sustained"
    return 1700.0, "fallback sustained"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_seconds(t_local: float, world: int, device: str = "cuda") -> float:
    """Seconds of the whole job: the slowest rank's mean step time (max over ranks)."""
    if world <= 1:
        return float(t_local)
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(t_job: float, world: int) -> float:
    """Solves per second over all ranks: each rank solves its own replica (no data exchange)."""
    return world / t_job


def rotation_flops(hist, n):
    # Step 11 on V only: the solver keeps just W's newest k_b columns, which it recomputes
    return sum(2.0 * n * h.k_old * h.k_act for h in hist)


# A slice product with S digit slices runs S (S + 1) / 2 bf16 x bf16 -> f32 tensor-core
# products (pairs s + t < S; see csrc/ozaki.cu): 36 for S = 8 (float64-accurate), 21 for S = 6
# (the mixed path's Step-11 rotation).
def slice_pairs(S):
    return S * (S + 1) // 2


# DRAM bytes (read + write) per launch of the filter SpMM (spmm_axpby_kernel<float, 4>, one
# residual-form step) on the 1M-node SBM: dram__bytes_read.sum + dram__bytes_write.sum of three
# interior filter steps in a one-pass ncu capture of the current kernel (470.4 + 68.6 MB); to
# be set back to None whenever the kernel changes
FILTER_TRAFFIC_BYTES = {"sbm1m": 539_027_029}


def filter_model_bytes(n, nnz, b, m, iters, s):
    """Compulsory bytes of the filter SpMM per solve by the scope table's model: per step
    4 (N + 1) + nnz (4 + s) + 3 N b s (the first step of a filter 2 N b s), m steps per filter,
    one filter per outer iteration; s = value and vector element bytes."""
    csr = 4.0 * (n + 1) + nnz * (4.0 + s)
    per_filter = m * csr + (2 + 3 * (m - 1)) * n * b * s
    return iters * per_filter

# Slice pairs per float64-equivalent flop, by path.  On the mixed path the first DGKS
# projection's Gram product runs on 4 slices (10 pairs) and Step 11 on 6 (21 pairs); Step 8
# stays at 8 slices (36 pairs) on both paths.
MIXED_LOW_SLICES = 4


def orth_flops(hist, n, b):
    return sum(8.0 * n * h.k_orth * b + 4.0 * n * b * b for h in hist)


def h_flops(hist, n, b):
    return sum(2.0 * n * h.k_old * b for h in hist)


def pair_work(name, hist, n, b, mixed):
    """Sum over the iterations of flops x slice pairs of each product of a component."""
    full = slice_pairs(8)
    low = slice_pairs(MIXED_LOW_SLICES)
    if name == "rotation":
        return (slice_pairs(6) if mixed else full) * rotation_flops(hist, n)
    if name == "orthonormalisation":
        p1 = low if mixed else full
        return sum(p1 * 2.0 * n * h.k_orth * b
                   + full * (6.0 * n * h.k_orth * b + 4.0 * n * b * b) for h in hist)
    return full * h_flops(hist, n, b)


def run_ours(args):
    import torch
    import torch.distributed as tdist
    import paper_2212_04443_gb300 as P
    import synth

    world, rank, local = dist()
    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl")
    hbm_peak, peak_kind = load_peaks()
    t_gen = time.perf_counter()
    w = synth.workload(args.workload)
    t_gen = time.perf_counter() - t_gen
    g = w["graph"]
    k, b, m, act, tol = w["k"], w["b"], w["m"], w["act_max"], w["tol"]
    prec = P.PREC_MIXED if args.precision == "mixed" else P.PREC_FP64
    H = P.Handle()
    src = torch.from_numpy(g.src).cuda()
    dst = torch.from_numpy(g.dst).cuda()
    kind = P.LAPLACIAN_COMBINATORIAL if w.get("kind") == "combinatorial" else \
        P.LAPLACIAN_NORMALIZED
    A = H.build_laplacian(g.n, src, dst, kind=kind)
    bounds, lz_steps = w.get("bounds"), w.get("lanczos_steps", 0)
    V0 = torch.from_numpy(synth.gaussian_block(g.n, b, w["v0_seed"])).cuda()
    evals = torch.zeros(k, dtype=torch.float64, device="cuda")
    evecs = torch.zeros((g.n, k), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    dense_path = args.dense_path

    def solve(precision, record=True):
        return H.solve(A, k, b, m, act, tol, v_init=V0, precision=precision,
                       record_history=record, evals=evals, evecs=evecs, itmax=200,
                       dense_path=dense_path, bounds=bounds, lanczos_steps=lz_steps)

    for _ in range(args.warmup):
        solve(prec)
    torch.cuda.synchronize()
    if world > 1:
        tdist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    times, infos, hists = [], [], []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, info = solve(prec)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        infos.append(info)
        hists.append(H.history())
    torch.cuda.synchronize()
    if world > 1:
        tdist.barrier()
    clk = clocks.stop()
    t_mean = job_seconds(float(np.mean(times)), world)
    info = infos[-1]
    hist = hists[-1]
    ok = all(i.status == 0 and i.max_rel_resid <= tol * 1.0001 for i in infos)
    ev_mixed = evals.cpu().numpy().copy()

    # ---- per-component roofline of the timed solve
    n = g.n
    sx = 4.0 if prec == P.PREC_MIXED else 8.0
    model_bytes = filter_model_bytes(n, A.nnz, b, m, info.iters, sx)
    comp = {
        "filter": dict(ms=info.ms["filter"], work=model_bytes, bound="hbm", unit="GB/s"),
        "rotation": dict(ms=info.ms["rot"], work=rotation_flops(hist, n), unit="TFLOP/s"),
        "orthonormalisation": dict(ms=info.ms["orth"], work=orth_flops(hist, n, b), unit="TFLOP/s"),
        "rayleigh_quotient": dict(ms=info.ms["h"], work=h_flops(hist, n, b), unit="TFLOP/s"),
    }
    tensor_path = dense_path != 1
    bf16_peak, bf16_kind = load_bf16_peak()
    for name, c in comp.items():
        s = c["ms"] / 1e3
        if c["unit"] == "GB/s":
            c["achieved"] = c["work"] / s / 1e9 if s > 0 else 0.0
            c["peak"] = hbm_peak
        elif tensor_path:
            # products executed as slice-pair bf16 tensor-core products: the method's own
            # float64 flop rate beside the rate of bf16 slice work it costs
            pw = pair_work(name, hist, n, b, prec == P.PREC_MIXED)
            c["bound"] = "tensor"
            c["slice_pairs"] = round(pw / c["work"], 2) if c["work"] > 0 else 0.0
            c["method_fp64_tflops"] = c["work"] / s / 1e12 if s > 0 else 0.0
            c["achieved"] = pw / s / 1e12 if s > 0 else 0.0
            c["peak"] = bf16_peak
        else:
            c["bound"] = "alu"
            c["achieved"] = c["work"] / s / 1e12 if s > 0 else 0.0
            c["peak"] = FP64_PEAK_TFLOPS
    # The metric names the filter SpMM: its rate by the scope table's compulsory-byte model
    # (CSR once, each row of X once, the previous block once, the output once) is the line's
    # roofline; the residual-form operands the kernel also streams are reported beside it.
    fc = comp["filter"]
    ms_f = fc["ms"]
    kern_bytes = info.filter_bytes
    launches = info.iters * m
    roofline = {
        "kernel": "spmm_axpby_kernel<float, 4> (filter SpMM, Algorithm 3)" if prec == P.PREC_MIXED
        else "spmm_axpby_kernel<double, 2> (filter SpMM, Algorithm 3)",
        "bound": "hbm", "achieved": round(fc["achieved"], 1), "peak": hbm_peak, "unit": "GB/s",
        "frac": round(fc["achieved"] / hbm_peak, 4),
        "traffic": (FILTER_TRAFFIC_BYTES.get(args.workload) if prec == P.PREC_MIXED else None),
        "model_bytes_per_launch": round(model_bytes / launches),
        "launch_us": round(ms_f * 1e3 / launches, 2),
        "note": "achieved = scope-table model bytes of the filter's m SpMM steps per outer "
                "iteration / the filter's device time (CUDA events around each filter)",
        "peak_source": f"{peak_kind} HBM copy rate (MEASURED_PEAKS.json)"}
    filter_roof = {"bound": "hbm", "model_gbs": round(fc["achieved"], 1),
                   "model_frac": round(fc["achieved"] / hbm_peak, 4),
                   "model_bytes_per_solve": model_bytes,
                   "kernel_bytes_per_solve": kern_bytes,
                   "kernel_gbs": round(kern_bytes / (ms_f / 1e3) / 1e9, 1) if ms_f > 0 else 0.0,
                   "kernel_bytes_note": "what the kernel streams: also the residual operand R and "
                                        "the own-row read of X (residual-form filter)",
                   "ms_per_solve": round(ms_f, 3), "peak": hbm_peak, "peak_source": peak_kind}
    breakdown = {kk: round(v, 3) for kk, v in info.ms.items()}
    components = {kk: {key: (round(v, 3) if isinstance(v, float) else v)
                       for key, v in c.items() if key != "work"} for kk, c in comp.items()}

    out = {}
    # ---- float64 path beside it
    if not args.no_fp64_compare and prec == P.PREC_MIXED and rank == 0:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, i64 = solve(P.PREC_FP64)
        e1.record(stream)
        e1.synchronize()
        ev64 = evals.cpu().numpy()
        out["fp64_path"] = {"seconds": round(e0.elapsed_time(e1) / 1e3, 4), "iters": i64.iters,
                            "status": i64.status, "max_rel_resid": i64.max_rel_resid,
                            "max_abs_eig_diff_mixed_vs_fp64": float(np.abs(ev_mixed - ev64).max()),
                            "breakdown_ms": {kk: round(v, 2) for kk, v in i64.ms.items()}}
    # ---- end to end through the host-buffer entry point
    if not args.no_e2e:
        rp = A.rowptr.cpu().pin_memory()
        ci = A.colidx.cpu().pin_memory()
        va = A.val.cpu().pin_memory()
        v0h = V0.cpu().pin_memory()
        evh = torch.zeros(k, dtype=torch.float64).pin_memory()
        evech = torch.zeros((n, k), dtype=torch.float64).pin_memory()
        rpn, cin, van, v0n = rp.numpy(), ci.numpy(), va.numpy(), v0h.numpy()
        e2e_times = []
        for it in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            H.solve_host(n, rpn, cin, van, k, b, m, act, tol, precision=prec, v_init=v0n,
                         evals=evh.numpy(), evecs=evech.numpy(), bounds=bounds,
                         lanczos_steps=lz_steps)
            torch.cuda.synchronize()
            e2e_times.append(time.perf_counter() - t0)
        h2d = rp.numel() * 4 + ci.numel() * 4 + va.numel() * 8 + v0h.numel() * 8
        d2h = k * 8 + n * k * 8
        out["e2e"] = {"value": round(min(e2e_times), 4), "unit": "s",
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    # ---- Step 1 bounds (Sec. 2): the k-step Lanczos estimate timed alone
    if bounds == "lanczos" and rank == 0:
        steps = lz_steps or 20
        H.lanczos_bounds(A, steps, 0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lo, hi, _, _ = H.lanczos_bounds(A, steps, 0)
        e1.record(stream)
        e1.synchronize()
        t_lz = e0.elapsed_time(e1) / 1e3
        out["bounds"] = {"mode": "lanczos", "steps": steps, "lowb": lo, "upperb": hi,
                         "seconds": round(t_lz, 5), "in_solve": [info.lowb, info.upperb]}
    # ---- Algorithm 1, Steps 4-5 on the eigenvectors (graphs with planted labels)
    if not args.no_cluster and rank == 0 and g.labels is not None:
        try:
            out["spectral_clustering"] = cluster_leg(
                H, g, evecs, stream, (clk or {}).get("sm_max_mhz") or 2070.0,
                with_oracle=(world == 1 and not args.no_cpu_baseline))
        except Exception as exc:   # report, keep the main line
            out["spectral_clustering"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
    # ---- learned start block (network trained on graphs of the workload's family)
    if not args.no_warm_start and rank == 0 and args.workload in WARM_FAMILIES:
        try:
            out["warm_start"] = warm_start_leg(args.workload, prec, stream)
        except Exception as exc:   # report, keep the main line
            out["warm_start"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
    # ---- many small graphs in one call (the batch512 workload)
    if not args.no_batched and rank == 0 and not args.workload.startswith("batch"):
        try:
            out["batched"] = batched_leg(prec, args.workers, args.batch_graphs)
        except Exception as exc:   # report, keep the main line
            out["batched"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
    # ---- CPU oracle on a bounded sample (rank 0, one GPU only)
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        out["cpu_baseline"] = cpu_baseline(args.workload, info.iters)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(t_mean, 4), "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_mean * 1e3, 2),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 filter / f64" if prec == P.PREC_MIXED else "f64",
            "data": "synthetic (seeded graph, device-built Laplacian, Gaussian V0)",
            "config": {"workload": f"{w['desc']}; k={k} b={b} m={m} act_max={act} tol={tol:g}",
                       "generation_s": round(t_gen, 1),
                       "n": g.n, "nnz": A.nnz, "k": k, "b": b, "m": m, "act_max": act,
                       "precision": args.precision, "dense_path": dense_path,
                       "l2": f"inputs larger than L2 (CSR {A.nnz * 12 / 1e9:.2f} GB, basis "
                             f"{g.n * (act + 2 * b) * 8 / 1e9:.1f} GB)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "iters": info.iters, "converged": ok, "max_rel_resid": info.max_rel_resid,
            "solves_per_s_all_gpus": round(replica_throughput(t_mean, world), 4),
            "roofline": roofline, "filter_spmm": filter_roof, "breakdown_ms": breakdown,
            "components": components,
            "gpu_launches": int(sum(i.launches for i in infos)),
            "clocks": clk,
        }
        line.update(out)
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()


def partition_scores(a, b):
    """Adjusted Rand index (Hubert and Arabie, 1985) and NMI (arithmetic normalisation) of
    two labelings, from their contingency table."""
    _, ia = np.unique(a, return_inverse=True)
    _, ib = np.unique(b, return_inverse=True)
    M = np.zeros((ia.max() + 1, ib.max() + 1))
    np.add.at(M, (ia, ib), 1.0)
    pairs = lambda x: x * (x - 1.0) / 2.0
    s_ij, s_a, s_b = pairs(M).sum(), pairs(M.sum(1)).sum(), pairs(M.sum(0)).sum()
    exp = s_a * s_b / pairs(M.sum())
    ari = 1.0 if 0.5 * (s_a + s_b) == exp else (s_ij - exp) / (0.5 * (s_a + s_b) - exp)
    P = M / M.sum()
    pa, pb = P.sum(1), P.sum(0)
    nz = P > 0
    mi = np.sum(P[nz] * np.log(P[nz] / np.outer(pa, pb)[nz]))
    h = -np.sum(pa * np.log(pa)) - np.sum(pb * np.log(pb))
    return float(ari), float(1.0 if h == 0 else 2 * mi / h)


def cluster_leg(H, g, evecs, stream, sm_max_mhz, with_oracle):
    """Row normalisation, farthest-first seeding and Lloyd's k-means on the solver's
    eigenvectors (one bchdav_spectral_cluster call, then each stage alone), scored against the
    planted labels.  The assignment rounds are bound by float32 issue: 3 operations per node,
    centroid and dimension against 128 float32 lanes per SM at the maximum SM clock."""
    import torch
    import synth
    n, k = evecs.shape
    c = int(np.unique(g.labels).size)
    first = synth.kmeans_first(n, 0)

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    V = evecs.contiguous()
    H.spectral_cluster(V, c, first)                       # warm-up
    runs = [timed(lambda: H.spectral_cluster(V, c, first)) for _ in range(3)]
    (lab, _, _, rounds), t_all = min(runs, key=lambda r: r[1])
    # each stage alone (outputs allocated by a first call, then timed; best of two)
    Xt = H.row_normalize(V)
    t_norm = min(timed(lambda: H.row_normalize(V, Xt))[1] for _ in range(2))
    seeds = H.kmeans_seed(Xt, c, first)
    t_seed = min(timed(lambda: H.kmeans_seed(Xt, c, first))[1] for _ in range(2))
    H.kmeans(Xt, seeds, 100)
    lloyd = [timed(lambda: H.kmeans(Xt, seeds, 100)) for _ in range(2)]
    (lab2, _, r2), t_lloyd = min(lloyd, key=lambda r: r[1])
    same = bool(torch.equal(lab, lab2))
    ari, nmi = partition_scores(lab.cpu().numpy(), g.labels)
    ops = 3.0 * n * c * k * r2
    sms = torch.cuda.get_device_properties(evecs.device).multi_processor_count
    peak = sms * 128 * sm_max_mhz * 1e6 / 1e12
    ach = ops / t_lloyd / 1e12
    out = {"clusters": c, "dim": k, "rounds": rounds, "ari": round(ari, 6), "nmi": round(nmi, 6),
           "seconds": round(t_all, 5), "stages_s": {"row_normalize": round(t_norm, 5),
                                                    "seeding": round(t_seed, 5),
                                                    "lloyd": round(t_lloyd, 5)},
           "stages_agree": same,
           "row_normalize_gbs": round(n * k * 12 / t_norm / 1e9, 1),
           "seeding_gbs": round((c - 1) * n * (4 * k + 8) / t_seed / 1e9, 1),
           "roofline": {"kernel": "km_assign_all_kernel (Lloyd rounds, whole bchdav_kmeans call)",
                        "bound": "alu", "achieved": round(ach, 3), "peak": round(peak, 2),
                        "unit": "Tops/s (float32)", "frac": round(ach / peak, 4),
                        "traffic": None,
                        "peak_source": f"{sms} SMs x 128 float32 lanes x maximum SM clock "
                                       f"({sm_max_mhz:.0f} MHz)"}}
    if with_oracle:   # the cpu_baseline leg: the oracle as it stands, on a bounded sample
        from oracle import cluster as OC
        rows = np.sort(synth.rng(77).choice(n, min(n, 20000), replace=False))
        Vs = V[torch.from_numpy(rows).cuda()].cpu().numpy()
        t0 = time.perf_counter()
        _, _, r_o, _ = OC.spectral_cluster(Vs, c, 0)
        t_o = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": t_o / rows.size / max(r_o, 1),
                               "unit": "s per node and Lloyd round", "cores": 1,
                               "kind": "oracle",
                               "sample": f"oracle.cluster.spectral_cluster on {rows.size} of {n} "
                                         f"rows: {t_o:.2f} s, {r_o} rounds"}
    return out


# Learned start block (Step 17's V_init): families, their training graphs and held-out graph.
# The network has at most 64 outputs, so the leg runs on smaller members of the family than
# the timed workload (k = 16).
WARM_FAMILIES = {
    "sbm1m": dict(desc="SBM, d_in = 16, d_out = 2, 16 clusters: trained on three 30,000-node "
                       "graphs (seeds 700-702), held out: a 60,000-node graph (seed 799)",
                  k=16, b=8, m=13, act=48,
                  train=lambda i: __import__("synth").sbm_edges(30000 + 1000 * i, 16, d_in=16.0,
                                                                d_out=2.0, seed=700 + i),
                  held=lambda: __import__("synth").sbm_edges(60000, 16, d_in=16.0, d_out=2.0,
                                                             seed=799)),
    "rmat24": dict(desc="R-MAT (0.57, 0.19, 0.19, 0.05), edge factor 16: trained on scales 11, "
                        "12, 12 (seeds 300-302), held out: scale 13 (seed 399)",
                   k=16, b=8, m=15, act=48,
                   train=lambda i: __import__("synth").rmat_edges([11, 12, 12][i], seed=300 + i),
                   held=lambda: __import__("synth").rmat_edges(13, seed=399)),
}


def warm_start_leg(workload, prec, stream):
    """Train the start-block network on solver eigenvectors of three graphs of the workload's
    family (two random-feature draws each), then solve a held-out graph of the family from the
    network's block and from random blocks (iterations and seconds of each)."""
    import torch
    import synth
    import paper_2212_04443_gb300 as P
    f = WARM_FAMILIES[workload]
    k, b, m, act, tol = f["k"], f["b"], f["m"], f["act"], 1e-8
    D_R, WIDTH, STEPS, LR = 14, 64, 150, 2e-3

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    Ht = P.Handle()
    As, Rs, Us = [], [], []
    for i in range(3):
        gt = f["train"](i)
        At = Ht.build_laplacian(gt.n, torch.from_numpy(gt.src).cuda(),
                                torch.from_numpy(gt.dst).cuda())
        _, Vt, _ = Ht.solve(At, k, b, m, act, tol, precision=prec, seed=i)
        for r in range(2):
            As.append(At)
            Us.append(Vt.contiguous())
            Rs.append(torch.from_numpy(synth.gnn_random_features(gt.n, D_R, 400 + 10 * i + r)).cuda())
    theta0 = torch.from_numpy(synth.gnn_init(D_R + 2, WIDTH, k, seed=11)).cuda()
    theta = theta0.clone()
    hist, t_train = timed(lambda: Ht.gnn_train(As, Rs, Us, theta, WIDTH, k, STEPS, LR))
    gh = f["held"]()
    Ah = Ht.build_laplacian(gh.n, torch.from_numpy(gh.src).cuda(), torch.from_numpy(gh.dst).cuda())
    R = torch.from_numpy(synth.gnn_random_features(gh.n, D_R, 499)).cuda()
    (V0, ritz), t_inf = timed(lambda: Ht.gnn_start_block(Ah, R, theta, WIDTH, k))
    _, ritz0 = Ht.gnn_start_block(Ah, R, theta0, WIDTH, k)
    (_, _, iw), t_warm = timed(lambda: Ht.solve(Ah, k, b, m, act, tol, precision=prec, v_init=V0))
    rnd = [timed(lambda s=s: Ht.solve(Ah, k, b, m, act, tol, precision=prec, seed=s))
           for s in range(3)]
    out = {"family": f["desc"], "k": k, "b": b, "train_steps": STEPS, "train_s": round(t_train, 3),
           "loss_first": round(float(hist[0].mean()), 4),
           "loss_last": round(float(hist[-1].mean()), 4),
           "ritz_mean_untrained": round(float(ritz0.mean()), 4),
           "ritz_mean_trained": round(float(ritz.mean()), 4), "inference_s": round(t_inf, 4),
           "warm": {"iters": iw.iters, "s": round(t_warm, 4), "status": iw.status},
           "random": [{"iters": r[0][2].iters, "s": round(r[1], 4), "status": r[0][2].status}
                      for r in rnd]}
    del As, Rs, Us, V0
    Ht.release_workspace()
    return out


def batched_leg(prec, workers, n_graphs=512):
    """bchdav_solve_batched on the batch512 workload (or its first n_graphs graphs, the same
    seeds): graphs/s of one warm call, per-graph latency percentiles, launches per graph."""
    import torch
    import synth
    import paper_2212_04443_gb300 as P
    graphs = _batch_head(n_graphs)
    Hb = P.Handle()
    As = [Hb.build_laplacian(g.n, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda())
          for g in graphs]
    cs = [int(g.labels.max()) + 1 for g in graphs]
    ks, bs = cs, [min(c, 8) for c in cs]

    def once():
        return Hb.solve_batched(As, ks, bs, [11] * n_graphs, [0] * n_graphs, 1e-8,
                                precision=prec, seed=0, workers=workers, itmax=200)

    once()
    torch.cuda.synchronize()
    l0 = P.launch_count()
    t0 = time.perf_counter()
    _, _, infos, per = once()
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    launches = P.launch_count() - l0
    out = {"workload": "batch512" if n_graphs == 512 else f"batch512 (first {n_graphs} graphs)",
           "graphs": n_graphs, "sum_n": int(sum(g.n for g in graphs)),
           "workers": workers, "graphs_per_s": round(n_graphs / t, 2), "seconds": round(t, 3),
           "latency_ms": {"p50": round(float(np.percentile(per, 50)), 2),
                          "p99": round(float(np.percentile(per, 99)), 2)},
           "launches_per_graph": round(launches / n_graphs, 1),
           "converged": all(i.status == 0 for i in infos)}
    Hb.release_workspace()
    return out


def _batch_head(n_graphs):
    """The first n_graphs graphs of synth.batch_sbm(512), generated without the rest."""
    import math
    import synth
    g = synth.rng(4)
    ns = np.floor(np.exp(g.uniform(math.log(2000), math.log(200000), 512))).astype(np.int64)
    cs = g.integers(4, 33, 512)
    return [synth.sbm_edges(int(ns[i]), int(cs[i]), d_in=12.0, d_out=1.5, seed=1000 + i)
            for i in range(n_graphs)]


def oracle_problem(w):
    """The workload's matrix as the oracle builds it, and its Step 1 bounds (None: [0, 2])."""
    import oracle
    from oracle import lanczos
    g = w["graph"]
    Asp = oracle.laplacian_csr(g.n, g.src, g.dst, kind=w.get("kind", "normalized")).scipy()
    bnd = None
    if w.get("bounds") == "lanczos":
        lo, hi, _, _ = lanczos.bounds(Asp, w.get("lanczos_steps") or 20, 0)
        bnd = (lo, hi)
    return Asp, bnd


def cpu_baseline(workload, gpu_iters, n_iter=2):
    """The oracle as it stands, timed on this host: the first n_iter outer iterations of the
    same solve, scaled by the iteration count of the full solve."""
    import oracle
    import synth
    w = synth.workload(workload)
    g = w["graph"]
    Asp, bnd = oracle_problem(w)
    V0 = synth.gaussian_block(g.n, w["b"], w["v0_seed"])
    t0 = time.perf_counter()
    oracle.bchdav(Asp, w["k"], w["b"], w["m"], w["act_max"], w["tol"], V_init=V0,
                  max_iters_run=n_iter, record=False, bounds=bnd)
    dt = time.perf_counter() - t0
    per_it = dt / n_iter
    golden = os.path.join(ROOT, "tests", "golden", f"oracle_{workload}.json")
    iters = gpu_iters
    if os.path.exists(golden):
        with open(golden) as f:
            iters = json.load(f).get("iters", gpu_iters)
    return {"value": round(per_it * iters, 2), "unit": "s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"first {n_iter} of {iters} outer iterations of the same solve "
                      f"({dt:.1f} s measured, {per_it:.2f} s/iteration, scaled by iterations; "
                      f"early iterations are the cheaper ones, so this underestimates)"}


def run_reference(args):
    """The oracle (the CPU restatement of the paper's method) on this host's cores."""
    world, rank, _ = dist()
    if rank != 0:
        return
    import oracle
    import synth
    w = synth.workload(args.workload)
    g = w["graph"]
    Asp, bnd = oracle_problem(w)
    V0 = synth.gaussian_block(g.n, w["b"], w["v0_seed"])
    golden = os.path.join(ROOT, "tests", "golden", f"oracle_{args.workload}.json")
    iters = None
    if os.path.exists(golden):
        with open(golden) as f:
            iters = json.load(f).get("iters")
    per = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.bchdav(Asp, w["k"], w["b"], w["m"], w["act_max"], w["tol"], V_init=V0,
                      max_iters_run=1, record=False, bounds=bnd)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            per.append(dt)
    per_it = float(np.mean(per))
    scale = iters or 1
    value = per_it * scale
    sample = (f"each step = outer iteration 1 of the solve ({per_it:.2f} s); value = that x "
              f"{scale} iterations of the full oracle solve")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": "s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(per_it * 1e3, 1), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded graph)",
        "config": {"workload": f"{w['desc']}; k={w['k']} b={w['b']} m={w['m']} "
                               f"act_max={w['act_max']} tol={w['tol']:g}"},
        "cpu_baseline": {"value": round(value, 2), "unit": "s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 2), "unit": "s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def run_batched(args):
    """Many independent SBM graphs solved side by side (bchdav_solve_batched): graphs/s for
    the whole batch and the per-graph latency distribution.  The graphs: sizes log-uniform in
    [2,000, 200,000], c uniform in [4, 32], intra-degree 12, inter-degree 1.5; k = c,
    b = min(c, 8), m = 11, act_max = max(5b, 30), tol = 1e-8; mixed precision."""
    import torch
    import paper_2212_04443_gb300 as P
    import synth

    n_graphs = int(args.workload.partition("@")[2] or 512)
    torch.cuda.set_device(0)
    t_gen = time.perf_counter()
    graphs = synth.batch_sbm(n_graphs)
    t_gen = time.perf_counter() - t_gen
    H = P.Handle()
    As = [H.build_laplacian(g.n, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda())
          for g in graphs]
    cs = [int(g.labels.max()) + 1 for g in graphs]
    ks, bs = cs, [min(c, 8) for c in cs]
    ms, acts = [11] * n_graphs, [0] * n_graphs
    prec = P.PREC_MIXED if args.precision == "mixed" else P.PREC_FP64

    def once():
        return H.solve_batched(As, ks, bs, ms, acts, 1e-8, precision=prec, seed=0,
                               workers=args.workers, itmax=200)

    for _ in range(args.warmup):
        once()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    times, lat, iters, ok, launches = [], [], [], True, 0
    for _ in range(args.steps):
        l0 = P.launch_count()
        t0 = time.perf_counter()
        ev, V, infos, per = once()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        launches += P.launch_count() - l0
        lat.extend(per.tolist())
        iters.extend(i.iters for i in infos)
        ok = ok and all(i.status == 0 and i.max_rel_resid <= 1e-8 * 1.0001 for i in infos)
    clk = clocks.stop()
    t = float(np.mean(times))
    line = {
        "metric": "graphs/s, batched SBM solves to rel. residual 1e-8", "value": round(n_graphs / t, 2),
        "unit": "graphs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t * 1e3, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 filter / f64" if prec == P.PREC_MIXED else "f64",
        "data": "synthetic (seeded SBM batch, device-built Laplacians, Philox start blocks)",
        "config": {"workload": f"{n_graphs} SBM graphs, N log-uniform [2000, 200000], c in [4, 32], "
                               "d_in=12 d_out=1.5; k=c b=min(c,8) m=11 act_max=max(5b,30) tol=1e-8",
                   "sum_n": int(sum(g.n for g in graphs)), "sum_nnz": int(sum(a.nnz for a in As)),
                   "workers": args.workers, "generation_s": round(t_gen, 1),
                   "l2": "graphs of up to 200,000 nodes: inputs of one graph fit in L2; the batch does not"},
        "converged": ok, "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 2),
                                        "p99": round(float(np.percentile(lat, 99)), 2),
                                        "max": round(float(np.max(lat)), 2)},
        "iters": {"mean": round(float(np.mean(iters)), 2), "max": int(np.max(iters))},
        "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith("batch"):
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
