"""GB300 (sm_103a) block Chebyshev-Davidson eigensolver for graph Laplacians.

Thin ctypes binding over the C-ABI library ``libbchdav.so`` (declared in
``include/bchdav.h``).  Every numerical step runs in the library's CUDA
kernels; this module only marshals arguments.  PyTorch supplies device
memory and the current CUDA stream.  Importing works without a GPU; any call
that needs the library raises if it was not built or cannot be loaded (there is
no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

__all__ = [
    "lib", "build", "Handle", "DeviceCSR", "BchdavError", "SolveInfo", "IterRecord",
    "PREC_FP64", "PREC_MIXED", "EXPORTED_SYMBOLS", "launch_count", "LAPLACIAN_NORMALIZED",
    "LAPLACIAN_COMBINATORIAL", "BOUNDS_NORMALIZED", "BOUNDS_GIVEN", "BOUNDS_LANCZOS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libbchdav.so")

PREC_FP64 = 0
PREC_MIXED = 1
LAPLACIAN_NORMALIZED = 0      # Eq. (1)
LAPLACIAN_COMBINATORIAL = 1   # D - S
BOUNDS_NORMALIZED, BOUNDS_GIVEN, BOUNDS_LANCZOS = 0, 1, 2

STATUS = {0: "ok", 1: "not converged", -1: "invalid argument", -2: "invalid CSR",
          -3: "out of device memory", -4: "CUDA error", -5: "non-finite value",
          -6: "device wait timed out"}

EXPORTED_SYMBOLS = [
    "bchdav_create", "bchdav_destroy", "bchdav_set_stream", "bchdav_status_string",
    "bchdav_last_error", "bchdav_build_laplacian", "bchdav_free_csr", "bchdav_copy_csr", "bchdav_check_csr",
    "bchdav_solve", "bchdav_solve_host", "bchdav_history", "bchdav_filter", "bchdav_spmm", "bchdav_spmm_dd",
    "bchdav_orthonormalize", "bchdav_gram", "bchdav_rotate", "bchdav_eigh",
    "bchdav_eigh_noalloc", "bchdav_solve_batched", "bchdav_set_batch_workers",
    "bchdav_launch_count", "bchdav_gnn_n_params", "bchdav_gnn_forward", "bchdav_gnn_loss_grad",
    "bchdav_gnn_train", "bchdav_gnn_start_block", "bchdav_release_workspace",
    "bchdav_row_normalize", "bchdav_kmeans_seed", "bchdav_kmeans", "bchdav_spectral_cluster",
    "bchdav_build_laplacian_kind", "bchdav_lanczos_bounds", "bchdav_set_memory_limit",
    "bchdav_workspace_bytes",
]


def launch_count() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().bchdav_launch_count())


class BchdavError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class CSRStruct(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("colidx", C.c_void_p), ("val", C.c_void_p), ("val_f32", C.c_void_p)]


class OptsStruct(C.Structure):
    _fields_ = [("dim_max", C.c_int32), ("itmax", C.c_int32), ("precision", C.c_int32),
                ("dense_path", C.c_int32), ("seed", C.c_uint64), ("v_init", C.c_void_p),
                ("k_init", C.c_int32), ("ld_v_init", C.c_int32), ("record_history", C.c_int32),
                ("bounds", C.c_int32), ("lowb", C.c_double), ("upperb", C.c_double),
                ("lanczos_steps", C.c_int32), ("reserved3", C.c_int32)]


class InfoStruct(C.Structure):
    _fields_ = [("iters", C.c_int32), ("n_converged", C.c_int32), ("n_spmm", C.c_int32),
                ("n_replaced", C.c_int32), ("max_rel_resid", C.c_double),
                ("ms_total", C.c_double), ("ms_filter", C.c_double), ("ms_orth", C.c_double),
                ("ms_spmm_w", C.c_double), ("ms_h", C.c_double), ("ms_eig", C.c_double),
                ("ms_rot", C.c_double), ("ms_resid", C.c_double), ("ms_other", C.c_double),
                ("filter_bytes", C.c_double), ("filter_ms_kernels", C.c_double),
                ("n_kernel_launches", C.c_int64), ("status", C.c_int32), ("reserved2", C.c_int32),
                ("lowb", C.c_double), ("upperb", C.c_double)]


class IterStruct(C.Structure):
    _fields_ = [("it", C.c_int32), ("k_c", C.c_int32), ("e_c", C.c_int32), ("k_act", C.c_int32),
                ("k_sub", C.c_int32), ("k_old", C.c_int32), ("n_rep", C.c_int32),
                ("k_orth", C.c_int32), ("low_nwb", C.c_double), ("max_resid", C.c_double),
                ("min_resid", C.c_double)]


_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    from .build import build as _build
    return _build(force=force, verbose=verbose)


def lib() -> C.CDLL:
    """Load libbchdav.so (building it first if sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    from .build import build as _build, needs_build
    if needs_build():
        _build()
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"CUDA library missing: {_LIB_PATH}")
    L = C.CDLL(_LIB_PATH)
    i32, i64, u64, d, p = C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.c_void_p
    sig = {
        "bchdav_create": (i32, [C.POINTER(p), p]),
        "bchdav_destroy": (i32, [p]),
        "bchdav_set_stream": (i32, [p, p]),
        "bchdav_set_memory_limit": (i32, [p, u64]),
        "bchdav_workspace_bytes": (u64, [p]),
        "bchdav_status_string": (C.c_char_p, [i32]),
        "bchdav_last_error": (C.c_char_p, [p]),
        "bchdav_build_laplacian": (i32, [p, i32, i64, p, p, C.POINTER(CSRStruct)]),
        "bchdav_free_csr": (i32, [p, C.POINTER(CSRStruct)]),
        "bchdav_copy_csr": (i32, [p, C.POINTER(CSRStruct), p, p, p, p]),
        "bchdav_check_csr": (i32, [p, C.POINTER(CSRStruct)]),
        "bchdav_solve": (i32, [p, C.POINTER(CSRStruct), i32, i32, i32, i32, d,
                               C.POINTER(OptsStruct), p, p, C.POINTER(InfoStruct)]),
        "bchdav_solve_host": (i32, [p, i32, i64, p, p, p, i32, i32, i32, i32, d,
                                    C.POINTER(OptsStruct), p, p, C.POINTER(InfoStruct)]),
        "bchdav_history": (i32, [p, C.POINTER(IterStruct), i32]),
        "bchdav_solve_batched": (i32, [p, i32, C.POINTER(CSRStruct), p, p, p, p, d,
                                       C.POINTER(OptsStruct), p, p, C.POINTER(InfoStruct), p]),
        "bchdav_set_batch_workers": (i32, [p, i32]),
        "bchdav_launch_count": (i64, []),
        "bchdav_release_workspace": (i32, [p]),
        "bchdav_gnn_n_params": (i64, [i32, i32, i32]),
        "bchdav_gnn_forward": (i32, [p, C.POINTER(CSRStruct), p, i32, p, i32, i32, p]),
        "bchdav_gnn_loss_grad": (i32, [p, C.POINTER(CSRStruct), p, i32, p, i32, i32, p, d, p,
                                       p, p]),
        "bchdav_gnn_train": (i32, [p, i32, C.POINTER(CSRStruct), p, i32, p, i32, i32, p, i32, d,
                                   d, p]),
        "bchdav_gnn_start_block": (i32, [p, C.POINTER(CSRStruct), p, i32, p, i32, i32, p, p]),
        "bchdav_filter": (i32, [p, C.POINTER(CSRStruct), p, i32, i32, i32, d, d, d, i32, p, i32]),
        "bchdav_spmm": (i32, [p, C.POINTER(CSRStruct), p, i32, i32, p, i32]),
        "bchdav_spmm_dd": (i32, [p, C.POINTER(CSRStruct), p, i32, i32, p, i32]),
        "bchdav_orthonormalize": (i32, [p, i32, p, i32, i32, p, i32, i32, u64, d,
                                        C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
        "bchdav_eigh": (i32, [p, i32, p, i32, p, p, i32]),
        "bchdav_rotate": (i32, [p, i32, p, i32, i32, p, i32, i32, i32]),
        "bchdav_gram": (i32, [p, i32, p, i32, i32, p, i32, i32, p, i32]),
        "bchdav_eigh_noalloc": (i32, [i32, p, i32, p, p, i32, p]),
        "bchdav_row_normalize": (i32, [p, i32, i32, p, i64, p, i64]),
        "bchdav_build_laplacian_kind": (i32, [p, i32, i64, p, p, i32, C.POINTER(CSRStruct)]),
        "bchdav_lanczos_bounds": (i32, [p, C.POINTER(CSRStruct), i32, u64, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), p, p, C.POINTER(C.c_int32)]),
        "bchdav_kmeans_seed": (i32, [p, i32, i32, p, i64, i32, i32, p]),
        "bchdav_kmeans": (i32, [p, i32, i32, p, i64, i32, p, i32, p, p, C.POINTER(C.c_int32)]),
        "bchdav_spectral_cluster": (i32, [p, i32, i32, p, i64, i32, i32, i32, p, p, p,
                                          C.POINTER(C.c_int32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _set_bounds(opts, bounds, lanczos_steps):
    if bounds is None:
        opts.bounds = BOUNDS_NORMALIZED
    elif isinstance(bounds, str):
        if bounds != "lanczos":
            raise ValueError(f"bounds: {bounds!r}")
        opts.bounds = BOUNDS_LANCZOS
        opts.lanczos_steps = lanczos_steps
    else:
        opts.bounds = BOUNDS_GIVEN
        opts.lowb, opts.upperb = float(bounds[0]), float(bounds[1])


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


@dataclass
class DeviceCSR:
    """The Laplacian in CSR form, held in torch CUDA tensors."""
    n: int
    rowptr: "object"   # int32 [n+1]
    colidx: "object"   # int32 [nnz]
    val: "object"      # float64 [nnz]
    val_f32: "object" = None  # float32 [nnz] or None

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    def struct(self) -> CSRStruct:
        return CSRStruct(self.n, self.nnz, _ptr(self.rowptr), _ptr(self.colidx), _ptr(self.val),
                         _ptr(self.val_f32))


@dataclass
class SolveInfo:
    status: int
    iters: int
    n_converged: int
    n_spmm: int
    n_replaced: int
    max_rel_resid: float
    ms: dict
    filter_bytes: float
    filter_ms: float
    launches: int
    lowb: float = 0.0
    upperb: float = 2.0


@dataclass
class IterRecord:
    it: int
    k_c: int
    e_c: int
    k_act: int
    k_sub: int
    k_old: int
    n_rep: int
    k_orth: int
    low_nwb: float
    max_resid: float
    min_resid: float


class Handle:
    """A library handle bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream=None):
        import torch
        self.L = lib()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self._stream = int(stream)
        h = C.c_void_p()
        st = self.L.bchdav_create(C.byref(h), C.c_void_p(self._stream))
        if st != 0:
            raise BchdavError(st, self.L.bchdav_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.bchdav_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=(0,)):
        if st not in allow:
            raise BchdavError(st, self.L.bchdav_last_error(self.h).decode())
        return st

    def set_memory_limit(self, nbytes: int):
        """Cap the device workspace this handle may hold (0 removes the cap)."""
        self._check(self.L.bchdav_set_memory_limit(self.h, int(nbytes)))

    def workspace_bytes(self) -> int:
        return int(self.L.bchdav_workspace_bytes(self.h))

    def set_stream(self, stream):
        self._stream = int(stream)
        self._check(self.L.bchdav_set_stream(self.h, C.c_void_p(self._stream)))

    # ---- Eq. (1)
    def build_laplacian(self, n: int, src, dst, kind: int = LAPLACIAN_NORMALIZED) -> DeviceCSR:
        """A = I - D^{-1/2} S D^{-1/2} (or with kind=LAPLACIAN_COMBINATORIAL, D - S) from int32
        CUDA edge tensors (library-built CSR)."""
        import torch
        cs = CSRStruct()
        self._check(self.L.bchdav_build_laplacian_kind(self.h, n, int(src.numel()), _ptr(src),
                                                       _ptr(dst), kind, C.byref(cs)))
        nnz = int(cs.nnz)
        dev = src.device
        # copy into torch-owned tensors, then release the library's arrays
        rowptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
        colidx = torch.empty(nnz, dtype=torch.int32, device=dev)
        val = torch.empty(nnz, dtype=torch.float64, device=dev)
        val32 = torch.empty(nnz, dtype=torch.float32, device=dev)
        torch.cuda.synchronize(dev)
        try:
            self._check(self.L.bchdav_copy_csr(self.h, C.byref(cs), _ptr(rowptr), _ptr(colidx),
                                               _ptr(val), _ptr(val32)))
        finally:
            self.L.bchdav_free_csr(self.h, C.byref(cs))
        return DeviceCSR(n, rowptr, colidx, val, val32)

    def check_csr(self, A: DeviceCSR):
        cs = A.struct()
        return self._check(self.L.bchdav_check_csr(self.h, C.byref(cs)), allow=(0, -2))

    # ---- Algorithm 2
    def solve(self, A: DeviceCSR, k: int, b: int, m: int, act_max: int, tol: float, *,
              v_init=None, precision: int = PREC_FP64, dim_max: int = 0, itmax: int = 0,
              seed: int = 0, record_history: bool = False, evals=None, evecs=None,
              dense_path: int = 0, bounds=None, lanczos_steps: int = 0):
        """bounds: None (the normalized Laplacian's [0, 2]), (lowb, upperb), or "lanczos"."""
        import torch
        dev = A.rowptr.device
        if evals is None:
            evals = torch.zeros(k, dtype=torch.float64, device=dev)
        if evecs is None:
            evecs = torch.zeros((A.n, k), dtype=torch.float64, device=dev)
        opts = OptsStruct()
        opts.dim_max = dim_max
        opts.itmax = itmax
        opts.precision = precision
        opts.seed = seed
        opts.dense_path = dense_path
        opts.record_history = 1 if record_history else 0
        _set_bounds(opts, bounds, lanczos_steps)
        if v_init is not None:
            assert v_init.dtype == torch.float64 and v_init.is_cuda and v_init.stride(1) == 1
            opts.v_init = _ptr(v_init)
            opts.k_init = v_init.shape[1]
            opts.ld_v_init = v_init.stride(0)
        info = InfoStruct()
        cs = A.struct()
        st = self.L.bchdav_solve(self.h, C.byref(cs), k, b, m, act_max, tol, C.byref(opts),
                                 _ptr(evals), _ptr(evecs), C.byref(info))
        self._check(st, allow=(0, 1))
        return evals, evecs, self._info(st, info)

    def solve_host(self, n, rowptr, colidx, val, k, b, m, act_max, tol, *, precision=PREC_FP64,
                   seed=0, evals=None, evecs=None, v_init=None, bounds=None, lanczos_steps=0):
        """End-to-end call with host (numpy) arrays: copies in, solves, copies out."""
        import numpy as np
        if evals is None:
            evals = np.zeros(k)
        if evecs is None:
            evecs = np.zeros((n, k))
        opts = OptsStruct()
        opts.precision = precision
        opts.seed = seed
        _set_bounds(opts, bounds, lanczos_steps)
        if v_init is not None:
            v_init = np.ascontiguousarray(v_init, dtype=np.float64)
            opts.v_init = v_init.ctypes.data
            opts.k_init = v_init.shape[1]
            opts.ld_v_init = v_init.shape[1]
        info = InfoStruct()
        st = self.L.bchdav_solve_host(self.h, n, int(colidx.shape[0]), rowptr.ctypes.data,
                                      colidx.ctypes.data, val.ctypes.data, k, b, m, act_max, tol,
                                      C.byref(opts), evals.ctypes.data, evecs.ctypes.data,
                                      C.byref(info))
        self._check(st, allow=(0, 1))
        return evals, evecs, self._info(st, info)

    def solve_batched(self, As, k, b, m, act_max, tol, *, precision: int = PREC_MIXED,
                      seed: int = 0, workers: int = 8, dense_path: int = 0, itmax: int = 0):
        """Independent solves of many graphs (lists of equal length; act_max entries 0 take the
        default).  Returns (evals list, evecs list, [SolveInfo], per-graph ms numpy array)."""
        import numpy as np
        import torch
        n = len(As)
        evals = [torch.zeros(int(k[i]), dtype=torch.float64, device=As[i].rowptr.device)
                 for i in range(n)]
        evecs = [torch.zeros((As[i].n, int(k[i])), dtype=torch.float64,
                             device=As[i].rowptr.device) for i in range(n)]
        arr = (CSRStruct * n)(*[a.struct() for a in As])
        i32a = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.int32))
        ka, ba, ma, aa = i32a(k), i32a(b), i32a(m), i32a(act_max)
        pe = np.array([_ptr(t) for t in evals], dtype=np.uint64)
        pv = np.array([_ptr(t) for t in evecs], dtype=np.uint64)
        infos = (InfoStruct * n)()
        ms = np.zeros(n, dtype=np.float32)
        opts = OptsStruct()
        opts.precision = precision
        opts.seed = seed
        opts.dense_path = dense_path
        opts.itmax = itmax
        self._check(self.L.bchdav_set_batch_workers(self.h, workers))
        st = self.L.bchdav_solve_batched(self.h, n, arr, ka.ctypes.data, ba.ctypes.data,
                                         ma.ctypes.data, aa.ctypes.data, tol, C.byref(opts),
                                         pe.ctypes.data, pv.ctypes.data, infos, ms.ctypes.data)
        self._check(st, allow=(0, 1))
        return evals, evecs, [self._info(infos[i].status, infos[i]) for i in range(n)], ms

    def release_workspace(self):
        """Free the handle's device workspace (reallocated by the next call)."""
        self._check(self.L.bchdav_release_workspace(self.h))

    # ---- learned start block (network feeding V_init)
    def gnn_n_params(self, d_r: int, width: int, k: int) -> int:
        return int(self.L.bchdav_gnn_n_params(d_r, width, k))

    @staticmethod
    def _f32(t):
        import torch
        assert t.dtype == torch.float32 and t.is_cuda and t.is_contiguous()
        return _ptr(t)

    def gnn_forward(self, A: DeviceCSR, R, theta, width: int, k: int):
        import torch
        Z = torch.empty((A.n, k), dtype=torch.float32, device=A.rowptr.device)
        cs = A.struct()
        self._check(self.L.bchdav_gnn_forward(self.h, C.byref(cs), self._f32(R), R.shape[1],
                                              self._f32(theta), width, k, _ptr(Z)))
        return Z

    def gnn_loss_grad(self, A: DeviceCSR, R, theta, U, width: int, k: int, ridge: float = 1e-6):
        import torch
        grad = torch.empty_like(theta)
        Z = torch.empty((A.n, k), dtype=torch.float32, device=A.rowptr.device)
        loss = C.c_double(0.0)
        cs = A.struct()
        assert U.dtype == torch.float64 and U.is_contiguous() and U.shape == (A.n, k)
        self._check(self.L.bchdav_gnn_loss_grad(self.h, C.byref(cs), self._f32(R), R.shape[1],
                                                self._f32(theta), width, k, _ptr(U), ridge,
                                                _ptr(grad), C.addressof(loss), _ptr(Z)))
        return loss.value, grad, Z

    def gnn_train(self, As, Rs, Us, theta, width: int, k: int, steps: int, lr: float,
                  ridge: float = 1e-4):
        """Adam on theta (in place); returns the loss history (steps x graphs)."""
        import numpy as np
        n = len(As)
        arr = (CSRStruct * n)(*[a.struct() for a in As])
        pr = np.array([self._f32(r) for r in Rs], dtype=np.uint64)
        pu = np.array([_ptr(u) for u in Us], dtype=np.uint64)
        hist = np.zeros((steps, n))
        self._check(self.L.bchdav_gnn_train(self.h, n, arr, pr.ctypes.data, Rs[0].shape[1],
                                            pu.ctypes.data, width, k, self._f32(theta), steps,
                                            lr, ridge, hist.ctypes.data))
        return hist

    def gnn_start_block(self, A: DeviceCSR, R, theta, width: int, k: int):
        import torch
        V0 = torch.empty((A.n, k), dtype=torch.float64, device=A.rowptr.device)
        ritz = torch.empty(k, dtype=torch.float64, device=A.rowptr.device)
        cs = A.struct()
        self._check(self.L.bchdav_gnn_start_block(self.h, C.byref(cs), self._f32(R), R.shape[1],
                                                  self._f32(theta), width, k, _ptr(V0),
                                                  _ptr(ritz)))
        return V0, ritz

    # ---- Sec. 2: spectrum bounds by k-step Lanczos
    def lanczos_bounds(self, A: DeviceCSR, steps: int = 20, seed: int = 0):
        """(lowb, upperb, alpha, beta) of the k-step estimate (numpy arrays of the steps done)."""
        import numpy as np
        lo, hi = C.c_double(0.0), C.c_double(0.0)
        alpha, beta = np.zeros(steps), np.zeros(steps)
        done = C.c_int32(0)
        cs = A.struct()
        self._check(self.L.bchdav_lanczos_bounds(self.h, C.byref(cs), steps, seed, C.byref(lo),
                                                 C.byref(hi), alpha.ctypes.data,
                                                 beta.ctypes.data, C.byref(done)))
        return lo.value, hi.value, alpha[:done.value].copy(), beta[:done.value].copy()

    # ---- Algorithm 1, Steps 4-5: spectral clustering
    def row_normalize(self, V, Xt=None):
        """Transposed float32 features (dim x n) of the float64 row-major block V (n x dim)."""
        import torch
        assert V.dtype == torch.float64 and V.is_cuda and V.stride(1) == 1
        n, dim = V.shape
        if Xt is None:
            Xt = torch.empty((dim, n), dtype=torch.float32, device=V.device)
        self._check(self.L.bchdav_row_normalize(self.h, n, dim, _ptr(V), V.stride(0), _ptr(Xt),
                                                Xt.stride(0)))
        return Xt

    def kmeans_seed(self, Xt, n_clusters: int, first: int):
        import torch
        dim, n = Xt.shape
        seeds = torch.empty(n_clusters, dtype=torch.int32, device=Xt.device)
        self._check(self.L.bchdav_kmeans_seed(self.h, n, dim, self._f32r(Xt), Xt.stride(0),
                                              n_clusters, first, _ptr(seeds)))
        return seeds

    def kmeans(self, Xt, seeds, max_rounds: int = 100):
        """(labels int32 [n], centroids float64 [c, dim], rounds)."""
        import torch
        dim, n = Xt.shape
        c = int(seeds.numel())
        assert seeds.dtype == torch.int32 and seeds.is_cuda
        labels = torch.empty(n, dtype=torch.int32, device=Xt.device)
        cent = torch.empty((c, dim), dtype=torch.float64, device=Xt.device)
        r = C.c_int32(0)
        self._check(self.L.bchdav_kmeans(self.h, n, dim, self._f32r(Xt), Xt.stride(0), c,
                                         _ptr(seeds), max_rounds, _ptr(labels), _ptr(cent),
                                         C.byref(r)))
        return labels, cent, r.value

    def spectral_cluster(self, V, n_clusters: int, first: int, max_rounds: int = 100):
        """Steps 4-5 on the eigenvector block V (n x dim float64): (labels, centroids, seeds,
        rounds)."""
        import torch
        assert V.dtype == torch.float64 and V.is_cuda and V.stride(1) == 1
        n, dim = V.shape
        labels = torch.empty(n, dtype=torch.int32, device=V.device)
        cent = torch.empty((n_clusters, dim), dtype=torch.float64, device=V.device)
        seeds = torch.empty(n_clusters, dtype=torch.int32, device=V.device)
        r = C.c_int32(0)
        self._check(self.L.bchdav_spectral_cluster(self.h, n, dim, _ptr(V), V.stride(0),
                                                   n_clusters, first, max_rounds, _ptr(labels),
                                                   _ptr(cent), _ptr(seeds), C.byref(r)))
        return labels, cent, seeds, r.value

    @staticmethod
    def _f32r(t):
        import torch
        assert t.dtype == torch.float32 and t.is_cuda and t.stride(1) == 1
        return _ptr(t)

    def _info(self, st, info) -> SolveInfo:
        ms = dict(total=info.ms_total, filter=info.ms_filter, orth=info.ms_orth,
                  spmm_w=info.ms_spmm_w, h=info.ms_h, eig=info.ms_eig, rot=info.ms_rot,
                  resid=info.ms_resid, other=info.ms_other)
        return SolveInfo(st, info.iters, info.n_converged, info.n_spmm, info.n_replaced,
                         info.max_rel_resid, ms, info.filter_bytes, info.filter_ms_kernels,
                         info.n_kernel_launches, info.lowb, info.upperb)

    def history(self):
        n = self.L.bchdav_history(self.h, None, 0)
        arr = (IterStruct * max(n, 1))()
        self.L.bchdav_history(self.h, arr, n)
        return [IterRecord(r.it, r.k_c, r.e_c, r.k_act, r.k_sub, r.k_old, r.n_rep, r.k_orth,
                           r.low_nwb, r.max_resid, r.min_resid) for r in arr[:n]]

    # ---- single steps
    def filter(self, A: DeviceCSR, X, m: int, a: float, upb: float, a0: float,
               precision: int = PREC_FP64, Y=None):
        import torch
        if Y is None:
            Y = torch.empty_like(X)
        cs = A.struct()
        self._check(self.L.bchdav_filter(self.h, C.byref(cs), _ptr(X), X.stride(0), X.shape[1], m,
                                         a, upb, a0, precision, _ptr(Y), Y.stride(0)))
        return Y

    def spmm(self, A: DeviceCSR, X, Y=None):
        import torch
        if Y is None:
            Y = torch.empty_like(X)
        cs = A.struct()
        self._check(self.L.bchdav_spmm(self.h, C.byref(cs), _ptr(X), X.stride(0), X.shape[1],
                                       _ptr(Y), Y.stride(0)))
        return Y

    def spmm_dd(self, A: DeviceCSR, X, Y=None):
        """Y = A X by the mixed path's double-float product (Steps 7 and 12)."""
        import torch
        if Y is None:
            Y = torch.empty_like(X)
        cs = A.struct()
        self._check(self.L.bchdav_spmm_dd(self.h, C.byref(cs), _ptr(X), X.stride(0), X.shape[1],
                                          _ptr(Y), Y.stride(0)))
        return Y

    def orthonormalize(self, V, X, *, seed: int = 0, tau_dep: float = 1e-10, rep_counter: int = 0):
        """In place on X; returns (n_replaced, new rep_counter)."""
        k = 0 if V is None else V.shape[1]
        rc = C.c_int64(rep_counter)
        nr = C.c_int32(0)
        self._check(self.L.bchdav_orthonormalize(
            self.h, X.shape[0], _ptr(V), (V.stride(0) if V is not None else 1), k, _ptr(X),
            X.stride(0), X.shape[1], seed, tau_dep, C.byref(rc), C.byref(nr)))
        return nr.value, rc.value

    def gram(self, A, B, dense_path: int = 0):
        """A^T B for row-major CUDA float64 blocks with the same number of rows."""
        import torch
        out = torch.empty((A.shape[1], B.shape[1]), dtype=torch.float64, device=A.device)
        self._check(self.L.bchdav_gram(self.h, A.shape[0], _ptr(A), A.stride(0), A.shape[1],
                                       _ptr(B), B.stride(0), B.shape[1], _ptr(out), dense_path))
        return out

    def rotate(self, V, Y, nb: int, dense_path: int = 0):
        """In place: V[:, :nb] = V[:, :k] @ Y[:, :nb] (k = Y.shape[0])."""
        k = Y.shape[0]
        self._check(self.L.bchdav_rotate(self.h, V.shape[0], _ptr(V), V.stride(0), k, _ptr(Y),
                                         Y.stride(0), nb, dense_path))
        return V

    def eigh(self, H):
        import torch
        n = H.shape[0]
        D = torch.empty(n, dtype=torch.float64, device=H.device)
        Y = torch.empty((n, n), dtype=torch.float64, device=H.device)
        self._check(self.L.bchdav_eigh(self.h, n, _ptr(H), H.stride(0), _ptr(D), _ptr(Y),
                                       Y.stride(0)))
        return D, Y
