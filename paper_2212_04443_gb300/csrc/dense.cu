// Tall-skinny dense FP64 kernels of Algorithm 2: Gram products V^T X (Step 6
// and Step 8), the update X -= V C (Step 6), the in-place subspace rotation
// V <- V Y (Step 11), column norms, block copies and small H updates.
//
// On GB300 FP64 FMA runs at ~1.2 TFLOP/s (2 per clock per SM), 1/58 of the
// FP32 rate, so these kernels are bound by the FP64 pipe, not by memory or
// shared memory: each keeps enough independent FMAs in flight per warp and
// stages the operand rows once in shared memory.  All cross-CTA reductions
// are two-stage with a fixed summation order (bitwise reproducible).
#include "kernels.cuh"

namespace bchdav {

unsigned long long g_launches = 0;

// ---------------- Gram: partial[c] = A_c^T B_c ----------------
constexpr int kTnThreads = 256;
constexpr int kTnRows = 16;     // rows staged per tile
constexpr int kTnMaxOut = 32;   // outputs per thread per pass

int gemm_tn_chunks(int n) {
  int c = ceil_div(n, 2048);
  int cap = 2 * kSMs;
  if (c > cap) c = cap;
  return c < 1 ? 1 : c;
}

// sym (A = B, ka = kb): outputs enumerate the upper triangle p <= q and each is stored at
// (p, q) and (q, p) -- the same sums as computing both (fma is symmetric in its factors).
// MAXOUT outputs per thread per pass: 2 for small Gram matrices (few registers, several CTAs
// per SM), kTnMaxOut otherwise.
template <int MAXOUT>
__global__ void __launch_bounds__(kTnThreads) gemm_tn_partial_kernel(
    int n, const double* __restrict__ A, int lda, int ka, const double* __restrict__ B, int ldb,
    int kb, double* __restrict__ partial, int out0, int out_count, int sym) {
  extern __shared__ double sm[];
  double* sA = sm;                       // kTnRows x ka
  double* sB = sm + kTnRows * ka;        // kTnRows x kb
  const int t = threadIdx.x;
  const int chunk = blockIdx.x;
  const int rows_per = (n + gridDim.x - 1) / gridDim.x;
  const int r_begin = chunk * rows_per;
  const int r_end = min(n, r_begin + rows_per);
  double acc[MAXOUT];
  int pp[MAXOUT], qq[MAXOUT];
#pragma unroll
  for (int i = 0; i < MAXOUT; ++i) {
    acc[i] = 0.0;
    int o = out0 + t + i * kTnThreads;
    const int total = sym ? ka * (ka + 1) / 2 : ka * kb;
    if (o < out_count + out0 && o < total) {
      if (sym) {
        int p = 0;
        while (o >= ka - p) {
          o -= ka - p;
          ++p;
        }
        pp[i] = p;
        qq[i] = p + o;
      } else {
        pp[i] = o / kb;
        qq[i] = o - pp[i] * kb;
      }
    } else {
      pp[i] = -1;
      qq[i] = 0;
    }
  }
  for (int r0 = r_begin; r0 < r_end; r0 += kTnRows) {
    const int nr = min(kTnRows, r_end - r0);
    __syncthreads();
    for (int idx = t; idx < kTnRows * ka; idx += kTnThreads) {
      int r = idx / ka, c = idx - r * ka;
      sA[idx] = (r < nr) ? A[(size_t)(r0 + r) * lda + c] : 0.0;
    }
    for (int idx = t; idx < kTnRows * kb; idx += kTnThreads) {
      int r = idx / kb, c = idx - r * kb;
      sB[idx] = (r < nr) ? B[(size_t)(r0 + r) * ldb + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXOUT; ++i) {
      if (pp[i] >= 0) {
        double s = acc[i];
#pragma unroll 4
        for (int r = 0; r < kTnRows; ++r) s = fma(sA[r * ka + pp[i]], sB[r * kb + qq[i]], s);
        acc[i] = s;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < MAXOUT; ++i) {
    if (pp[i] >= 0) {
      partial[(size_t)chunk * ka * kb + pp[i] * kb + qq[i]] = acc[i];
      if (sym) partial[(size_t)chunk * ka * kb + qq[i] * kb + pp[i]] = acc[i];
    }
  }
}

cudaError_t launch_gemm_tn_partial(cudaStream_t st, int n, const double* A, int lda, int ka,
                                   const double* B, int ldb, int kb, double* partial,
                                   int n_chunks) {
  if (ka <= 0 || kb <= 0) return cudaSuccess;
  size_t smem = (size_t)kTnRows * (ka + kb) * sizeof(double);
  // A^T A: the upper triangle only (half the float64 multiply-adds), mirrored
  const int sym = (A == B && ka == kb && lda == ldb) ? 1 : 0;
  const int total = sym ? ka * (ka + 1) / 2 : ka * kb;
  if (total <= 2 * kTnThreads) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(gemm_tn_partial_kernel<2>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    gemm_tn_partial_kernel<2><<<n_chunks, kTnThreads, smem, st>>>(n, A, lda, ka, B, ldb, kb,
                                                                  partial, 0, total, sym);
    note_launch();
    return cudaGetLastError();
  }
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tn_partial_kernel<kTnMaxOut>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int per_pass = kTnThreads * kTnMaxOut;
  for (int out0 = 0; out0 < total; out0 += per_pass) {
    gemm_tn_partial_kernel<kTnMaxOut><<<n_chunks, kTnThreads, smem, st>>>(
        n, A, lda, ka, B, ldb, kb, partial, out0, min(per_pass, total - out0), sym);
    note_launch();
  }
  return cudaGetLastError();
}

// Second stage of the two-stage sums, in a fixed order: four running sums over the chunks
// c = 0, 1, 2, 3 (mod 4), then (s0 + s1) + (s2 + s3).  Four independent chains: a float64 add
// waits ~64 cycles for the one before it on GB300, so one chain over a few hundred chunks
// took 10-20 us.
__global__ void reduce_partials_kernel(const double* __restrict__ partial, int n_chunks, int count,
                                       double* __restrict__ out, double scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int c = 0;
  for (; c + 3 < n_chunks; c += 4) {
    s0 += partial[(size_t)c * count + i];
    s1 += partial[(size_t)(c + 1) * count + i];
    s2 += partial[(size_t)(c + 2) * count + i];
    s3 += partial[(size_t)(c + 3) * count + i];
  }
  if (c < n_chunks) s0 += partial[(size_t)c * count + i];
  if (c + 1 < n_chunks) s1 += partial[(size_t)(c + 1) * count + i];
  if (c + 2 < n_chunks) s2 += partial[(size_t)(c + 2) * count + i];
  out[i] = scale * ((s0 + s1) + (s2 + s3));
}

cudaError_t launch_reduce_partials(cudaStream_t st, const double* partial, int n_chunks, int count,
                                   double* out, double scale) {
  if (count <= 0) return cudaSuccess;
  reduce_partials_kernel<<<ceil_div(count, 256), 256, 0, st>>>(partial, n_chunks, count, out,
                                                               scale); note_launch();
  return cudaGetLastError();
}

// ---------------- row-tile GEMM: C = A(rows) * B ----------------
constexpr int kNnThreads = 256;
constexpr int kNnRows = 32;   // rows per CTA
constexpr int kNnCols = 64;   // output columns per pass
// thread t: column t % 64, rows (t / 64) + 4 i, i < 8

template <bool INPLACE>
__global__ void __launch_bounds__(kNnThreads) gemm_nn_kernel(
    int n, const double* __restrict__ A, int lda, int k, const double* __restrict__ B, int ldb,
    int nb, double* __restrict__ C, int ldc) {
  extern __shared__ double sA[];   // kNnRows x k
  const int t = threadIdx.x;
  const int r0 = blockIdx.x * kNnRows;
  const int nr = min(kNnRows, n - r0);
  for (int idx = t; idx < kNnRows * k; idx += kNnThreads) {
    int r = idx / k, c = idx - r * k;
    sA[idx] = (r < nr) ? A[(size_t)(r0 + r) * lda + c] : 0.0;
  }
  __syncthreads();
  const int cl = t % kNnCols;
  const int rg = t / kNnCols;   // 0..3
  for (int c0 = 0; c0 < nb; c0 += kNnCols) {
    const int col = c0 + cl;
    double acc[kNnRows / 4];
#pragma unroll
    for (int i = 0; i < kNnRows / 4; ++i) acc[i] = 0.0;
    if (col < nb) {
      for (int kk = 0; kk < k; ++kk) {
        double bv = __ldg(B + (size_t)kk * ldb + col);
#pragma unroll
        for (int i = 0; i < kNnRows / 4; ++i) acc[i] = fma(sA[(rg + 4 * i) * k + kk], bv, acc[i]);
      }
#pragma unroll
      for (int i = 0; i < kNnRows / 4; ++i) {
        int r = rg + 4 * i;
        if (r < nr) {
          double* p = C + (size_t)(r0 + r) * ldc + col;
          if (INPLACE) *p = acc[i];
          else *p = *p - acc[i];
        }
      }
    }
  }
}

template <bool INPLACE>
static cudaError_t launch_nn(cudaStream_t st, int n, const double* A, int lda, int k,
                             const double* B, int ldb, int nb, double* C, int ldc) {
  if (n <= 0 || nb <= 0) return cudaSuccess;
  if (k <= 0) {
    return cudaSuccess;   // C -= 0 ; in-place with k = 0 has nothing to rotate
  }
  size_t smem = (size_t)kNnRows * k * sizeof(double);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gemm_nn_kernel<INPLACE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  gemm_nn_kernel<INPLACE><<<ceil_div(n, kNnRows), kNnThreads, smem, st>>>(n, A, lda, k, B, ldb, nb,
                                                                         C, ldc); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gemm_nn_sub(cudaStream_t st, int n, const double* A, int lda, int k,
                               const double* B, int ldb, int nb, double* C, int ldc) {
  return launch_nn<false>(st, n, A, lda, k, B, ldb, nb, C, ldc);
}

cudaError_t launch_gemm_nn_inplace(cudaStream_t st, int n, double* A, int lda, int k,
                                   const double* B, int ldb, int nb) {
  if (nb > k) return cudaErrorInvalidValue;
  return launch_nn<true>(st, n, A, lda, k, B, ldb, nb, A, lda);
}

// X(rows, 0:b) <- X(rows, 0:b) U in place, U upper triangular (b x b, ld ldu, b <= 64; the
// in-block step X R^{-1} of CholQR2).  Column j only needs U(0:j, j): the lanes of a warp are
// 32 rows sharing one column, so the shortened loop is the same for the whole warp; rows are
// staged with a padded stride (no shared-memory bank conflicts).  Each output sums k = 0..j in
// order, as the general kernel does over k = 0..b-1 with zeros beyond j.
constexpr int kTriRows = 32;

__global__ void __launch_bounds__(kNnThreads) gemm_tri_inplace_kernel(int n, double* __restrict__ X,
                                                                    int ldx, int b,
                                                                    const double* __restrict__ U,
                                                                    int ldu) {
  extern __shared__ double sx[];   // kTriRows x (b + 1)
  const int sp = b + 1;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int r0 = blockIdx.x * kTriRows;
  const int nr = min(kTriRows, n - r0);
  for (int idx = t; idx < kTriRows * b; idx += kNnThreads) {
    const int r = idx / b, c = idx - r * b;
    sx[r * sp + c] = r < nr ? X[(size_t)(r0 + r) * ldx + c] : 0.0;
  }
  __syncthreads();
  for (int col = warp; col < b; col += kNnThreads / 32) {
    double acc = 0.0;
    for (int kk = 0; kk <= col; ++kk) acc = fma(sx[lane * sp + kk], __ldg(U + (size_t)kk * ldu + col), acc);
    if (lane < nr) X[(size_t)(r0 + lane) * ldx + col] = acc;
  }
}

cudaError_t launch_gemm_tri_inplace(cudaStream_t st, int n, double* X, int ldx, int b,
                                    const double* U, int ldu) {
  if (n <= 0 || b <= 0) return cudaSuccess;
  if (b > 64) return cudaErrorInvalidValue;
  const size_t smem = (size_t)kTriRows * (b + 1) * sizeof(double);
  gemm_tri_inplace_kernel<<<ceil_div(n, kTriRows), kNnThreads, smem, st>>>(n, X, ldx, b, U, ldu);
  note_launch();
  return cudaGetLastError();
}

// ---------------- column sums of squares ----------------
// Per-CTA partial sums of squares of X's columns (fixed order: four running sums over the
// CTA's rows, then over its row groups), so that several loads and float64 chains are in flight
// per thread.
__global__ void col_sumsq_kernel(int n, const double* __restrict__ X, int ldx, int b,
                                 double* __restrict__ partial) {
  extern __shared__ double sh[];
  const int t = threadIdx.x;
  const int rpb = blockDim.x / b;
  const int rl = t / b, c = t - rl * b;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (rl < rpb) {
    const int step = gridDim.x * rpb;
    int row = blockIdx.x * rpb + rl;
    for (; row + 3 * step < n; row += 4 * step) {
      const double v0 = X[(size_t)row * ldx + c], v1 = X[(size_t)(row + step) * ldx + c];
      const double v2 = X[(size_t)(row + 2 * step) * ldx + c];
      const double v3 = X[(size_t)(row + 3 * step) * ldx + c];
      s0 = fma(v0, v0, s0);
      s1 = fma(v1, v1, s1);
      s2 = fma(v2, v2, s2);
      s3 = fma(v3, v3, s3);
    }
    for (; row < n; row += step) {
      const double v = X[(size_t)row * ldx + c];
      s0 = fma(v, v, s0);
    }
  }
  sh[t] = (rl < rpb) ? (s0 + s1) + (s2 + s3) : 0.0;
  __syncthreads();
  if (t < b) {
    double a0 = 0.0, a1 = 0.0;
    int q = 0;
    for (; q + 1 < rpb; q += 2) {
      a0 += sh[q * b + t];
      a1 += sh[(q + 1) * b + t];
    }
    if (q < rpb) a0 += sh[q * b + t];
    partial[(size_t)blockIdx.x * b + t] = a0 + a1;
  }
}

cudaError_t launch_col_sumsq_partial(cudaStream_t st, int n, const double* X, int ldx, int b,
                                     double* partial, int n_chunks) {
  if (b > 256 || b <= 0) return cudaErrorInvalidValue;
  col_sumsq_kernel<<<n_chunks, 256, 256 * sizeof(double), st>>>(n, X, ldx, b, partial); note_launch();
  return cudaGetLastError();
}

// ---------------- element-wise block utilities ----------------
__global__ void copy_block_kernel(int n, int w, const double* __restrict__ src, int lds,
                                  double* __restrict__ dst, int ldd) {
  long long total = (long long)n * w;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int r = (int)(i / w), c = (int)(i - (long long)r * w);
    dst[(size_t)r * ldd + c] = src[(size_t)r * lds + c];
  }
}

static int ew_grid(long long total) {
  long long g = (total + 255) / 256;
  long long cap = (long long)kSMs * 16;
  return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

cudaError_t launch_copy_block(cudaStream_t st, int n, int w, const double* src, int lds,
                              double* dst, int ldd) {
  if (n <= 0 || w <= 0) return cudaSuccess;
  copy_block_kernel<<<ew_grid((long long)n * w), 256, 0, st>>>(n, w, src, lds, dst, ldd); note_launch();
  return cudaGetLastError();
}

__global__ void shift_cols_left_kernel(int n, double* __restrict__ X, int ldx, int count,
                                       int shift) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    double* row = X + (size_t)r * ldx;
    for (int c0 = 0; c0 < count; c0 += 32) {
      int c = c0 + lane;
      double v = (c < count) ? row[c + shift] : 0.0;
      __syncwarp();
      if (c < count) row[c] = v;
      __syncwarp();
    }
  }
}

cudaError_t launch_shift_cols_left(cudaStream_t st, int n, double* X, int ldx, int count, int shift) {
  if (n <= 0 || count <= 0 || shift <= 0) return cudaSuccess;
  shift_cols_left_kernel<<<ew_grid((long long)n * 32), 256, 0, st>>>(n, X, ldx, count, shift); note_launch();
  return cudaGetLastError();
}

__global__ void gather_cols_kernel(int n, int w, const double* __restrict__ src, int lds,
                                   const int* __restrict__ perm, double* __restrict__ dst, int ldd) {
  long long total = (long long)n * w;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int r = (int)(i / w), c = (int)(i - (long long)r * w);
    dst[(size_t)r * ldd + c] = src[(size_t)r * lds + perm[c]];
  }
}

cudaError_t launch_gather_cols(cudaStream_t st, int n, int w, const double* src, int lds,
                               const int* perm, double* dst, int ldd) {
  if (n <= 0 || w <= 0) return cudaSuccess;
  gather_cols_kernel<<<ew_grid((long long)n * w), 256, 0, st>>>(n, w, src, lds, perm, dst, ldd); note_launch();
  return cudaGetLastError();
}

__global__ void f64_to_f32_kernel(int n, int w, const double* __restrict__ src, int lds,
                                  float* __restrict__ dst, int ldd) {
  long long total = (long long)n * w;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int r = (int)(i / w), c = (int)(i - (long long)r * w);
    dst[(size_t)r * ldd + c] = __double2float_rn(src[(size_t)r * lds + c]);
  }
}

__global__ void f32_to_f64_kernel(int n, int w, const float* __restrict__ src, int lds,
                                  double* __restrict__ dst, int ldd) {
  long long total = (long long)n * w;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int r = (int)(i / w), c = (int)(i - (long long)r * w);
    dst[(size_t)r * ldd + c] = (double)src[(size_t)r * lds + c];
  }
}

cudaError_t launch_f64_to_f32(cudaStream_t st, int n, int w, const double* src, int lds,
                              float* dst, int ldd) {
  if (n <= 0 || w <= 0) return cudaSuccess;
  f64_to_f32_kernel<<<ew_grid((long long)n * w), 256, 0, st>>>(n, w, src, lds, dst, ldd); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(cudaStream_t st, int n, int w, const float* src, int lds,
                              double* dst, int ldd) {
  if (n <= 0 || w <= 0) return cudaSuccess;
  f32_to_f64_kernel<<<ew_grid((long long)n * w), 256, 0, st>>>(n, w, src, lds, dst, ldd); note_launch();
  return cudaGetLastError();
}

__global__ void mixed_inputs_kernel(int n, int b, const double* __restrict__ X, int ldx,
                                    const double* __restrict__ R, int ldr,
                                    const int* __restrict__ src, float* __restrict__ Z0,
                                    float* __restrict__ R32, int ldo) {
  long long total = (long long)n * b;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int r = (int)(i / b), c = (int)(i - (long long)r * b);
    int s = src[c];
    float z = 0.f, rv = 0.f;
    if (s < 0) z = __double2float_rn(X[(size_t)r * ldx + c]);
    else rv = __double2float_rn(R[(size_t)r * ldr + s]);
    Z0[(size_t)r * ldo + c] = z;
    R32[(size_t)r * ldo + c] = rv;
  }
}

cudaError_t launch_mixed_inputs(cudaStream_t st, int n, int b, const double* X, int ldx,
                                const double* R, int ldr, const int* src, float* Z0, float* R32,
                                int ldo) {
  if (n <= 0 || b <= 0) return cudaSuccess;
  mixed_inputs_kernel<<<ew_grid((long long)n * b), 256, 0, st>>>(n, b, X, ldx, R, ldr, src, Z0,
                                                                R32, ldo); note_launch();
  return cudaGetLastError();
}

__global__ void f64_to_f32_vec_kernel(long long count, const double* __restrict__ src,
                                      float* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = __double2float_rn(src[i]);
}

cudaError_t launch_f64_to_f32_vec(cudaStream_t st, long long count, const double* src, float* dst) {
  if (count <= 0) return cudaSuccess;
  f64_to_f32_vec_kernel<<<ew_grid(count), 256, 0, st>>>(count, src, dst); note_launch();
  return cudaGetLastError();
}

__global__ void fill_random_col_kernel(int n, double* __restrict__ X, int ldx, int col,
                                       uint64_t seed, uint32_t stream, uint32_t vec) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    X[(size_t)r * ldx + col] = philox_pm_half(seed, stream, vec, (uint32_t)r);
}

cudaError_t launch_fill_random_col(cudaStream_t st, int n, double* X, int ldx, int col,
                                   uint64_t seed, uint32_t stream, uint32_t vec) {
  if (n <= 0) return cudaSuccess;
  fill_random_col_kernel<<<ew_grid(n), 256, 0, st>>>(n, X, ldx, col, seed, stream, vec); note_launch();
  return cudaGetLastError();
}

// ---------------- small matrices ----------------
__global__ void h_update_kernel(double* __restrict__ H, int ldh, const double* __restrict__ G,
                                int k_act, int b) {
  // G: k_act x b, G[i*b + j] = v_i^T w_j for the new column j (k_act - b + j)
  const int j0 = k_act - b;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k_act * b) return;
  int i = idx / b, j = idx - i * b;
  double g = G[idx];
  if (i < j0) {
    H[(size_t)i * ldh + j0 + j] = g;
    H[(size_t)(j0 + j) * ldh + i] = g;
  } else {
    int ii = i - j0;   // new-new block: (B + B^T)/2
    double gt = G[(size_t)(j0 + j) * b + ii];
    H[(size_t)i * ldh + j0 + j] = 0.5 * (g + gt);
  }
}

cudaError_t launch_h_update(cudaStream_t st, double* H, int ldh, const double* G, int k_act, int b) {
  int total = k_act * b;
  if (total <= 0) return cudaSuccess;
  h_update_kernel<<<ceil_div(total, 256), 256, 0, st>>>(H, ldh, G, k_act, b); note_launch();
  return cudaGetLastError();
}

__global__ void h_diag_kernel(double* __restrict__ H, int ldh, const double* __restrict__ d, int k,
                              int clear) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= clear * clear) return;
  int i = idx / clear, j = idx - i * clear;
  H[(size_t)i * ldh + j] = (i == j && i < k) ? d[i] : 0.0;
}

cudaError_t launch_h_diag(cudaStream_t st, double* H, int ldh, const double* d, int k, int clear) {
  if (clear <= 0) return cudaSuccess;
  h_diag_kernel<<<ceil_div((long long)clear * clear, 256), 256, 0, st>>>(H, ldh, d, k, clear); note_launch();
  return cudaGetLastError();
}

// G (b x b, row-major) = R^T R, R upper triangular; Rinv = R^{-1} (b <= 64, one block).
// flag = 1 when G is not numerically positive definite, when a pivot R_jj falls below
// rel_min * sqrt(G_jj) (a near dependence inside the block that this Cholesky route does not
// resolve) or below dep * norm0[j] (the dependence test of Step 6).
//
// Right-looking: after pivot j is taken, row j of R is formed in parallel and the trailing
// entries (i, k), j < i <= k, lose R_ji R_jk.  Each entry receives its updates in the order
// j = 0, 1, ... as one fused multiply-add each, the same arithmetic as the column-by-column
// (left-looking) form.  The inverse is built column by column: entry (i, j) of R^{-1} needs
// only earlier columns, so the rows of one column are computed in parallel.
constexpr int kCholThreads = 256;

__global__ void __launch_bounds__(kCholThreads) chol_inv_kernel(
    int b, const double* __restrict__ G, const double* __restrict__ norm0, double rel_min,
    double dep, double* __restrict__ Rinv, int* __restrict__ flag, double* __restrict__ colscale) {
  // trailing matrix, then R in the upper triangle; R^{-1} goes to the strict lower triangle,
  // transposed (entry (i, j), i < j, at row j, column i), and its diagonal to Rd
  __shared__ double A[64 * 65];
  __shared__ double Rd[64];
  __shared__ double Ds[64];   // equilibration D_jj (1 without colscale)
  __shared__ int s_bad;
  const int t = threadIdx.x;
  for (int j = t; j < b; j += kCholThreads) {
    double dj = 1.0;
    if (colscale != nullptr) {
      // 2^-e with 2^(e-1) <= sqrt(G_jj) < 2^e, so that the scaled diagonal lies in [1/4, 1)
      const double gjj = G[j * b + j];
      if (gjj > 0.0 && gjj < INFINITY) {
        const int e = (int)((__double_as_longlong(sqrt(gjj)) >> 52) & 0x7FF) - 1022;
        dj = (e > -1021 && e < 1022) ? __longlong_as_double((long long)(1023 - e) << 52) : 1.0;
      }
      colscale[j] = dj;
    }
    Ds[j] = dj;
  }
  __syncthreads();
  for (int idx = t; idx < b * b; idx += kCholThreads) {
    const int i = idx / b, k = idx - i * b;
    A[i * 65 + k] = G[idx] * Ds[i] * Ds[k];   // exact: powers of two
  }
  if (t == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (t == 0) {
      const double djj = A[j * 65 + j];
      int bad = 0;
      if (!(djj > 0.0)) {
        bad = 1;
      } else {
        const double rjj = sqrt(djj);
        if (!(rjj > rel_min * sqrt(G[j * b + j]) * Ds[j]) ||
            (norm0 && !(rjj > dep * norm0[j] * Ds[j])))
          bad = 1;
        A[j * 65 + j] = rjj;
      }
      s_bad = bad;
    }
    __syncthreads();
    if (s_bad) break;
    const double inv = 1.0 / A[j * 65 + j];
    for (int k = j + 1 + t; k < b; k += kCholThreads) A[j * 65 + k] *= inv;
    __syncthreads();
    // trailing update of the entries (i, k), j < i <= k
    const int m = b - j - 1;
    for (int idx = t; idx < m * m; idx += kCholThreads) {
      const int i = j + 1 + idx / m, k = j + 1 + idx % m;
      if (i <= k) A[i * 65 + k] = fma(-A[j * 65 + i], A[j * 65 + k], A[i * 65 + k]);
    }
    __syncthreads();
  }
  if (t == 0) *flag = s_bad;
  if (s_bad) return;
  // (R^{-1})_{ik} for i < k sits at A[k][i]; (R^{-1})_{ii} at Rd[i]
  for (int j = 0; j < b; ++j) {
    const double inv = 1.0 / A[j * 65 + j];
    if (t == 0) Rd[j] = inv;
    __syncthreads();
    for (int i = t; i < j; i += kCholThreads) {
      double v = Rd[i] * A[i * 65 + j];   // k = i
      for (int k = i + 1; k < j; ++k) v = fma(A[k * 65 + i], A[k * 65 + j], v);
      A[j * 65 + i] = -v * inv;
    }
    __syncthreads();
  }
  for (int idx = t; idx < b * b; idx += kCholThreads) {
    const int i = idx / b, j = idx - i * b;
    Rinv[idx] = (i < j) ? A[j * 65 + i] : (i == j ? Rd[i] : 0.0);
  }
}

cudaError_t launch_chol_inv(cudaStream_t st, int b, const double* G, const double* norm0,
                            double rel_min, double dep, double* Rinv, int* flag,
                            double* colscale) {
  if (b < 1 || b > 64) return cudaErrorInvalidValue;
  chol_inv_kernel<<<1, kCholThreads, 0, st>>>(b, G, norm0, rel_min, dep, Rinv, flag, colscale); note_launch();
  return cudaGetLastError();
}

__global__ void check_finite_kernel(int n, int w, const double* __restrict__ X, int ldx,
                                    int* __restrict__ flag) {
  long long total = (long long)n * w;
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int r = (int)(i / w), c = (int)(i - (long long)r * w);
    if (!isfinite(X[(size_t)r * ldx + c])) bad = 1;
  }
  if (bad) atomicOr(flag, 1);
}

cudaError_t launch_check_finite(cudaStream_t st, int n, int w, const double* X, int ldx, int* flag) {
  if (n <= 0 || w <= 0) return cudaSuccess;
  check_finite_kernel<<<ew_grid((long long)n * w), 256, 0, st>>>(n, w, X, ldx, flag); note_launch();
  return cudaGetLastError();
}

}  // namespace bchdav
