// CSR SpMM with a tall-skinny row-major block (Eq. (6)), fused with the
// three-term-recurrence epilogue of the Chebyshev filter (Algorithm 3) or with
// the residual norms of Algorithm 2, Step 12.
//
// Mapping: a group of TPR = b / VW consecutive threads owns one row; thread
// `lane` of the group owns VW consecutive columns (one 16-byte vector when
// VW * sizeof(T) == 16).  The group walks the row's nonzeros four at a time:
// colidx/val are read once per group (same address across the group, served
// as one request), the gathered rows of X are contiguous VW-vectors, so every
// nonzero costs exactly b * sizeof(T) bytes of gather traffic.  The epilogue
// reads X and Z at the row itself and writes Y once: compulsory bytes per
// launch are 4 (N + 1) + nnz (4 + sizeof(T)) + N b sizeof(T) (gathered X
// counted once) + 2 N b sizeof(T) (Z and Y).
#include "kernels.cuh"

namespace bchdav {

template <typename T, int VW>
struct VecT;
template <>
struct VecT<double, 1> { using type = double; };
template <>
struct VecT<double, 2> { using type = double2; };
template <>
struct VecT<float, 1> { using type = float; };
template <>
struct VecT<float, 2> { using type = float2; };
template <>
struct VecT<float, 4> { using type = float4; };

template <typename T, int VW>
__device__ __forceinline__ void ldv(const T* __restrict__ p, T (&v)[VW]) {
  using V = typename VecT<T, VW>::type;
  V x = __ldg(reinterpret_cast<const V*>(p));
  const T* e = reinterpret_cast<const T*>(&x);
#pragma unroll
  for (int i = 0; i < VW; ++i) v[i] = e[i];
}

template <typename T, int VW>
__device__ __forceinline__ void stv(T* __restrict__ p, const T (&v)[VW]) {
  using V = typename VecT<T, VW>::type;
  V x;
  T* e = reinterpret_cast<T*>(&x);
#pragma unroll
  for (int i = 0; i < VW; ++i) e[i] = v[i];
  *reinterpret_cast<V*>(p) = x;
}

template <typename T, int VW>
__device__ __forceinline__ void row_product(const int* __restrict__ colidx, const T* __restrict__ val,
                                            const T* __restrict__ X, int ldx, int c0, int start,
                                            int end, T (&acc)[VW]) {
  int k = start;
  for (; k + 3 < end; k += 4) {
    int j0 = __ldg(colidx + k), j1 = __ldg(colidx + k + 1);
    int j2 = __ldg(colidx + k + 2), j3 = __ldg(colidx + k + 3);
    T a0 = __ldg(val + k), a1 = __ldg(val + k + 1), a2 = __ldg(val + k + 2), a3 = __ldg(val + k + 3);
    T x0[VW], x1[VW], x2[VW], x3[VW];
    ldv<T, VW>(X + (size_t)j0 * ldx + c0, x0);
    ldv<T, VW>(X + (size_t)j1 * ldx + c0, x1);
    ldv<T, VW>(X + (size_t)j2 * ldx + c0, x2);
    ldv<T, VW>(X + (size_t)j3 * ldx + c0, x3);
#pragma unroll
    for (int i = 0; i < VW; ++i) {
      acc[i] = fma(a0, x0[i], acc[i]);
      acc[i] = fma(a1, x1[i], acc[i]);
      acc[i] = fma(a2, x2[i], acc[i]);
      acc[i] = fma(a3, x3[i], acc[i]);
    }
  }
  for (; k < end; ++k) {
    int j = __ldg(colidx + k);
    T a = __ldg(val + k);
    T x[VW];
    ldv<T, VW>(X + (size_t)j * ldx + c0, x);
#pragma unroll
    for (int i = 0; i < VW; ++i) acc[i] = fma(a, x[i], acc[i]);
  }
}

template <typename T, int VW>
__global__ void __launch_bounds__(256) spmm_axpby_kernel(
    int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
    const T* __restrict__ val, const T* __restrict__ X, int ldx, int b, T* __restrict__ Y, int ldy,
    const T* __restrict__ Z, int ldz, T alpha, T beta, T gamma, const T* __restrict__ R, int ldr,
    const T* __restrict__ delta, int tpr, int rpb) {
  const int t = threadIdx.x;
  const int rl = t / tpr;
  if (rl >= rpb) return;
  const int row = blockIdx.x * rpb + rl;
  if (row >= n) return;
  const int c0 = (t - rl * tpr) * VW;
  T acc[VW];
#pragma unroll
  for (int i = 0; i < VW; ++i) acc[i] = T(0);
  row_product<T, VW>(colidx, val, X, ldx, c0, __ldg(rowptr + row), __ldg(rowptr + row + 1), acc);
  T out[VW];
#pragma unroll
  for (int i = 0; i < VW; ++i) out[i] = alpha * acc[i];
  if (beta != T(0)) {
    T x[VW];
    ldv<T, VW>(X + (size_t)row * ldx + c0, x);
#pragma unroll
    for (int i = 0; i < VW; ++i) out[i] = fma(beta, x[i], out[i]);
  }
  if (Z != nullptr) {
    T z[VW];
    ldv<T, VW>(Z + (size_t)row * ldz + c0, z);
#pragma unroll
    for (int i = 0; i < VW; ++i) out[i] = fma(gamma, z[i], out[i]);
  }
  if (R != nullptr) {
    T r[VW];
    ldv<T, VW>(R + (size_t)row * ldr + c0, r);
#pragma unroll
    for (int i = 0; i < VW; ++i) out[i] = fma(__ldg(delta + c0 + i), r[i], out[i]);
  }
  stv<T, VW>(Y + (size_t)row * ldy + c0, out);
}

// VW = 1 variant with a ragged last group: any b, any alignment.
template <typename T>
__global__ void __launch_bounds__(256) spmm_axpby_scalar_kernel(
    int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
    const T* __restrict__ val, const T* __restrict__ X, int ldx, int b, T* __restrict__ Y, int ldy,
    const T* __restrict__ Z, int ldz, T alpha, T beta, T gamma, const T* __restrict__ R, int ldr,
    const T* __restrict__ delta, int tpr, int rpb) {
  const int t = threadIdx.x;
  const int rl = t / tpr;
  if (rl >= rpb) return;
  const int row = blockIdx.x * rpb + rl;
  if (row >= n) return;
  const int c0 = t - rl * tpr;
  if (c0 >= b) return;
  T acc[1] = {T(0)};
  row_product<T, 1>(colidx, val, X, ldx, c0, __ldg(rowptr + row), __ldg(rowptr + row + 1), acc);
  T out = alpha * acc[0];
  if (beta != T(0)) out = fma(beta, __ldg(X + (size_t)row * ldx + c0), out);
  if (Z != nullptr) out = fma(gamma, __ldg(Z + (size_t)row * ldz + c0), out);
  if (R != nullptr) out = fma(__ldg(delta + c0), __ldg(R + (size_t)row * ldr + c0), out);
  Y[(size_t)row * ldy + c0] = out;
}

template <typename T>
static int pick_vw(int b, const void* p1, int ld1, const void* p2, int ld2, const void* p3, int ld3) {
  const int cand[3] = {(int)(16 / sizeof(T)), (int)(8 / sizeof(T)), 1};
  for (int vw : cand) {
    if (vw < 1) continue;
    if (vw == 1) return 1;
    size_t bytes = (size_t)vw * sizeof(T);
    auto ok = [&](const void* p, int ld) {
      return p == nullptr || (((uintptr_t)p % bytes) == 0 && (ld % vw) == 0);
    };
    if (b % vw == 0 && ok(p1, ld1) && ok(p2, ld2) && ok(p3, ld3)) return vw;
  }
  return 1;
}

template <typename T>
cudaError_t launch_spmm_axpby(cudaStream_t st, int n, const int* rowptr, const int* colidx,
                              const T* val, const T* X, int ldx, int b, T* Y, int ldy,
                              const T* Z, int ldz, T alpha, T beta, T gamma, const T* R, int ldr,
                              const T* delta) {
  if (n <= 0 || b <= 0) return cudaSuccess;
  int vw = pick_vw<T>(b, X, ldx, Y, ldy, Z, ldz);
  if (R != nullptr && vw > 1 && (((uintptr_t)R % (vw * sizeof(T))) != 0 || ldr % vw != 0)) vw = 1;
  int tpr = (b + vw - 1) / vw;
  if (tpr > 256) return cudaErrorInvalidValue;
  int rpb = 256 / tpr;
  int threads = rpb * tpr;
  int grid = ceil_div(n, rpb);
  if (vw == 1) {
    spmm_axpby_scalar_kernel<T><<<grid, threads, 0, st>>>(n, rowptr, colidx, val, X, ldx, b, Y,
                                                          ldy, Z, ldz, alpha, beta, gamma, R, ldr, delta, tpr, rpb); note_launch();
  } else if (vw == 2) {
    spmm_axpby_kernel<T, 2><<<grid, threads, 0, st>>>(n, rowptr, colidx, val, X, ldx, b, Y, ldy,
                                                      Z, ldz, alpha, beta, gamma, R, ldr, delta,
                                                      tpr, rpb); note_launch();
  } else {
    if constexpr (sizeof(T) == 4) {
      spmm_axpby_kernel<T, 4><<<grid, threads, 0, st>>>(n, rowptr, colidx, val, X, ldx, b, Y, ldy,
                                                        Z, ldz, alpha, beta, gamma, R, ldr, delta,
                                                      tpr, rpb); note_launch();
    }
  }
  return cudaGetLastError();
}

template cudaError_t launch_spmm_axpby<double>(cudaStream_t, int, const int*, const int*,
                                               const double*, const double*, int, int, double*,
                                               int, const double*, int, double, double, double,
                                               const double*, int, const double*);
template cudaError_t launch_spmm_axpby<float>(cudaStream_t, int, const int*, const int*,
                                              const float*, const float*, int, int, float*, int,
                                              const float*, int, float, float, float, const float*,
                                              int, const float*);

// ---------------- residual norms (Step 12) ----------------
constexpr int kResidThreads = 256;

__global__ void __launch_bounds__(kResidThreads) spmm_resid_kernel(
    int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
    const double* __restrict__ val, const double* __restrict__ V, int ldv, int b,
    const double* __restrict__ d, double* __restrict__ partial, double* __restrict__ Rout,
    int ldr) {
  // one thread per (row, column); block covers rows_per_block rows of all b columns
  extern __shared__ double sh[];
  const int rpb = kResidThreads / b;
  const int t = threadIdx.x;
  const int rl = t / b;
  const int c = t - rl * b;
  double r2 = 0.0, v2 = 0.0;
  if (rl < rpb) {
    for (int row = blockIdx.x * rpb + rl; row < n; row += gridDim.x * rpb) {
      double acc[1] = {0.0};
      row_product<double, 1>(colidx, val, V, ldv, c, __ldg(rowptr + row), __ldg(rowptr + row + 1),
                             acc);
      double v = __ldg(V + (size_t)row * ldv + c);
      double r = fma(-__ldg(d + c), v, acc[0]);
      if (Rout != nullptr) Rout[(size_t)row * ldr + c] = r;
      r2 = fma(r, r, r2);
      v2 = fma(v, v, v2);
    }
  }
  // deterministic reduction over the rpb row slots of each column
  double* s_r = sh;
  double* s_v = sh + kResidThreads;
  s_r[t] = (rl < rpb) ? r2 : 0.0;
  s_v[t] = (rl < rpb) ? v2 : 0.0;
  __syncthreads();
  if (t < b) {
    double ar = 0.0, av = 0.0;
    for (int q = 0; q < rpb; ++q) {
      ar += s_r[q * b + t];
      av += s_v[q * b + t];
    }
    partial[(size_t)blockIdx.x * 2 * b + t] = ar;
    partial[(size_t)blockIdx.x * 2 * b + b + t] = av;
  }
}

int spmm_resid_max_parts(int n, int b) {
  int rpb = kResidThreads / (b > 0 ? b : 1);
  int g = ceil_div(n, rpb);
  return g < 4 * kSMs ? g : 4 * kSMs;
}

cudaError_t launch_spmm_resid(cudaStream_t st, int n, const int* rowptr, const int* colidx,
                              const double* val, const double* V, int ldv, int b,
                              const double* d, double* partial, int* n_parts, double* Rout,
                              int ldr) {
  if (b > kResidThreads || b <= 0) return cudaErrorInvalidValue;
  int grid = spmm_resid_max_parts(n, b);
  *n_parts = grid;
  spmm_resid_kernel<<<grid, kResidThreads, 2 * kResidThreads * sizeof(double), st>>>(
      n, rowptr, colidx, val, V, ldv, b, d, partial, Rout, ldr); note_launch();
  return cudaGetLastError();
}

}  // namespace bchdav
