// Float64-accurate tall-skinny products on the tensor cores (Steps 6 and 11 of
// Algorithm 2: X -= V C and V <- V Y), by error-free splitting of the
// operands into small-integer slices (Ozaki, Ogita, Oishi, Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 2012).
//
// Every row i of A (N x K) gets an exponent E_i with |a_ij| < 2^E_i, every
// column j of B (K x n) an exponent F_j; |a_ij| 2^-E_i is rounded to the
// nearest multiple of 2^-48 and written in balanced base-64 digits,
//     a_ij = 2^E_i  sum_{s=1..8} alpha^s_ij 2^{-6 s} + O(2^{E_i - 49}),
//     alpha^1 in {-64..64}, alpha^s in {-32..32} (s >= 2)
// (digits taken from the float64 bit pattern with integer operations; the
// rounding keeps the split unbiased), likewise b_jk with F_k, and
//     (A B)_ik = 2^{E_i + F_k} sum_{L=2..9} 2^{-6 L} sum_{s+t=L} (alpha^s beta^t)_ik
// where the terms with s + t > 9 (below 2^-54 relative) are dropped.  Each
// alpha^s beta^t is a bf16 x bf16 -> f32 tensor-core product of integers; a
// level sums at most 8 such products of K terms, each bounded by 64 * 64 when
// it holds a leading digit and 32 * 32 otherwise, so for K <= 448 the float32
// accumulation is exact (448 * (4096 + 2 * 2048 + 6 * 1024) < 2^24).  The
// eight level sums are combined in float64 in the epilogue.
//
// Products: legacy warp-level mma.sync m16n8k16 (bf16 in, f32 accumulate).
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace bchdav {

constexpr int kOzS = 8;          // slices
constexpr int kOzBits = 6;       // bits per slice
constexpr int kOzMaxK = 448;     // exactness bound of the per-level float32 sums
constexpr int kOzBM = 64;        // CTA tile rows
constexpr int kOzBN = 32;        // CTA tile columns
constexpr int kOzBK = 16;        // k step
constexpr int kOzRowStride = 24; // smem row stride (bf16) of a 16-wide k tile: conflict-free

// --- digit extraction ------------------------------------------------------
__device__ __forceinline__ int oz_exp_plus1(double a) {
  // e + 1 where |a| = 1.m * 2^e; very small (subnormal) values count as zero
  unsigned long long bits = (unsigned long long)__double_as_longlong(a);
  int ef = (int)((bits >> 52) & 0x7FF);
  return ef == 0 ? -100000 : ef - 1023 + 1;
}

// fixed-point magnitude F = round(|a| * 2^(48 - E)) (half up), F <= 2^48 when |a| < 2^E
__device__ __forceinline__ unsigned long long oz_fixed(double a, int E) {
  unsigned long long bits = (unsigned long long)__double_as_longlong(a);
  int ef = (int)((bits >> 52) & 0x7FF);
  if (ef == 0) return 0ull;
  unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;   // 53 bits
  int e = ef - 1023;
  int shift = 4 + E - e;   // |a| = mant 2^(e-52): F = mant 2^-(52 - 48 + E - e)
  if (shift >= 64) return 0ull;
  return (mant + (1ull << (shift - 1))) >> shift;   // shift >= 5 since |a| < 2^E
}

// balanced base-64 digits of F (8 digits, most significant first): d[0] in [0, 64],
// d[1..7] in [-32, 31]; sum_s d[s] 64^(7-s) = F
__device__ __forceinline__ void oz_digits(unsigned long long F, int (&d)[kOzS]) {
  long long X = (long long)F;
#pragma unroll
  for (int s = kOzS - 1; s >= 1; --s) {
    long long r = ((X + 32) & 63) - 32;
    d[s] = (int)r;
    X = (X - r) >> 6;
  }
  d[0] = (int)X;
}

__device__ __forceinline__ __nv_bfloat16 oz_bf16(int d, bool neg) {
  return __float2bfloat16_rn((float)(neg ? -d : d));   // |d| <= 64: exact
}

// Row exponents of A (N x K): E[i] = max_j (exponent(a_ij) + 1); 0 for zero rows.
__global__ void oz_row_exp_kernel(int n, const double* __restrict__ A, int lda, int K,
                                  int* __restrict__ E) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    int m = -100000;
    for (int j = lane; j < K; j += 32) m = max(m, oz_exp_plus1(A[(size_t)r * lda + j]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) E[r] = (m < -50000) ? 0 : m;
  }
}

// Slices of A: planes S x N x Kp (row-major, zero padded in k).
__global__ void oz_split_rows_kernel(int n, const double* __restrict__ A, int lda, int K, int Kp,
                                     const int* __restrict__ E, __nv_bfloat16* __restrict__ P) {
  const size_t plane = (size_t)n * Kp;
  const long long total = (long long)n * Kp;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / Kp), k = (int)(idx - (long long)r * Kp);
    const double a = (k < K) ? A[(size_t)r * lda + k] : 0.0;
    int d[kOzS];
    oz_digits(oz_fixed(a, E[r]), d);
    const bool neg = a < 0.0;
#pragma unroll
    for (int s = 0; s < kOzS; ++s) P[s * plane + idx] = oz_bf16(d[s], neg);
  }
}

// Column exponents and transposed slices of B (K x nb): planes S x nbp x Kp.
__global__ void oz_split_cols_kernel(int K, int nb, const double* __restrict__ B, int ldb, int Kp,
                                     int nbp, int* __restrict__ F_out, __nv_bfloat16* __restrict__ P) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const size_t plane = (size_t)nbp * Kp;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nbp; c += warps) {
    int m = -100000;
    if (c < nb)
      for (int k = lane; k < K; k += 32) m = max(m, oz_exp_plus1(B[(size_t)k * ldb + c]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int Ec = (m < -50000) ? 0 : m;
    if (lane == 0) F_out[c] = Ec;
    for (int k = lane; k < Kp; k += 32) {
      const double b = (c < nb && k < K) ? B[(size_t)k * ldb + c] : 0.0;
      int d[kOzS];
      oz_digits(oz_fixed(b, Ec), d);
      const bool neg = b < 0.0;
#pragma unroll
      for (int s = 0; s < kOzS; ++s) P[s * plane + (size_t)c * Kp + k] = oz_bf16(d[s], neg);
    }
  }
}

__device__ __forceinline__ void oz_mma(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

// C(rows, cols) = / -= A B from the slices.  CTA: 8 warps as 4 (rows) x 2 (cols), warp tile
// 16 x 16 (one m16 tile, two n8 tiles); k steps of 16 double-buffered through shared memory.
template <bool SUB>
__global__ void __launch_bounds__(256) oz_gemm_kernel(int n, int nb, int Kp, const __nv_bfloat16* __restrict__ PA,
                                                      const int* __restrict__ EA,
                                                      const __nv_bfloat16* __restrict__ PB, int nbp,
                                                      const int* __restrict__ EB,
                                                      double* __restrict__ C, int ldc) {
  extern __shared__ __align__(16) unsigned char oz_smem[];
  // sA[buf][s][row * kOzRowStride + k], sB likewise (73.7 KB: dynamic shared memory)
  auto sA = reinterpret_cast<__nv_bfloat16(*)[kOzS][kOzBM * kOzRowStride]>(oz_smem);
  auto sB = reinterpret_cast<__nv_bfloat16(*)[kOzS][kOzBN * kOzRowStride]>(
      oz_smem + sizeof(__nv_bfloat16) * 2 * kOzS * kOzBM * kOzRowStride);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int wm = warp & 3, wn = warp >> 2;
  const int r0 = blockIdx.x * kOzBM, c0 = blockIdx.y * kOzBN;
  const size_t planeA = (size_t)n * Kp, planeB = (size_t)nbp * Kp;
  const int g = lane >> 2, tig = lane & 3;

  auto load_stage = [&](int buf, int k0) {
    // A: S planes x 64 rows x 2 chunks of 16 B ; B: S planes x 32 rows x 2 chunks
    for (int q = t; q < kOzS * kOzBM * 2; q += 256) {
      const int s = q / (kOzBM * 2), rem = q - s * kOzBM * 2, row = rem >> 1, half = rem & 1;
      const int gr = r0 + row;
      __nv_bfloat16* dst = &sA[buf][s][row * kOzRowStride + half * 8];
      if (gr < n) cp_async16(dst, PA + s * planeA + (size_t)gr * Kp + k0 + half * 8);
      else *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
    }
    for (int q = t; q < kOzS * kOzBN * 2; q += 256) {
      const int s = q / (kOzBN * 2), rem = q - s * kOzBN * 2, row = rem >> 1, half = rem & 1;
      const int gc = c0 + row;
      __nv_bfloat16* dst = &sB[buf][s][row * kOzRowStride + half * 8];
      if (gc < nbp) cp_async16(dst, PB + s * planeB + (size_t)gc * Kp + k0 + half * 8);
      else *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
    }
    cp_async_commit();
  };

  float acc[kOzS][2][4];
#pragma unroll
  for (int L = 0; L < kOzS; ++L)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[L][j][e] = 0.f;

  const int nk = Kp / kOzBK;
  load_stage(0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    cp_async_wait0();
    __syncthreads();
    if (kt + 1 < nk) load_stage(buf ^ 1, (kt + 1) * kOzBK);
    // B fragments of all slices for the warp's two n8 tiles
    uint32_t bf[kOzS][2][2];
#pragma unroll
    for (int s = 0; s < kOzS; ++s)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const __nv_bfloat16* base = &sB[buf][s][(wn * 16 + j * 8 + g) * kOzRowStride];
        bf[s][j][0] = *reinterpret_cast<const uint32_t*>(base + tig * 2);
        bf[s][j][1] = *reinterpret_cast<const uint32_t*>(base + tig * 2 + 8);
      }
#pragma unroll
    for (int s = 0; s < kOzS; ++s) {
      uint32_t af[4];
      const __nv_bfloat16* base = &sA[buf][s][(wm * 16 + g) * kOzRowStride];
      af[0] = *reinterpret_cast<const uint32_t*>(base + tig * 2);
      af[1] = *reinterpret_cast<const uint32_t*>(base + 8 * kOzRowStride + tig * 2);
      af[2] = *reinterpret_cast<const uint32_t*>(base + tig * 2 + 8);
      af[3] = *reinterpret_cast<const uint32_t*>(base + 8 * kOzRowStride + tig * 2 + 8);
#pragma unroll
      for (int tt = 0; tt < kOzS; ++tt) {
        if (s + tt < kOzS) {   // levels s + tt + 2 <= 9
          oz_mma(acc[s + tt][0], af, bf[tt][0]);
          oz_mma(acc[s + tt][1], af, bf[tt][1]);
        }
      }
    }
  }
  // epilogue: combine the levels in float64 and scale by 2^(E_i + F_k)
#pragma unroll
  for (int j = 0; j < 2; ++j) {
#pragma unroll
    for (int hrow = 0; hrow < 2; ++hrow) {
      const int row = r0 + wm * 16 + g + hrow * 8;
      if (row >= n) continue;
      const int Er = EA[row];
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int col = c0 + wn * 16 + j * 8 + tig * 2 + cc;
        if (col >= nb) continue;
        const int base_exp = Er + EB[col];
        double v = 0.0;
#pragma unroll
        for (int L = kOzS - 1; L >= 0; --L) {
          const int ex = base_exp - kOzBits * (L + 2);
          const double scale =
              (ex > -1022) ? __longlong_as_double((long long)(ex + 1023) << 52) : 0.0;
          v = fma((double)acc[L][j][hrow * 2 + cc], scale, v);
        }
        double* p = C + (size_t)row * ldc + col;
        if (SUB) *p -= v;
        else *p = v;
      }
    }
  }
}

size_t ozaki_nn_work_bytes(int n, int K, int nb) {
  const size_t Kp = (size_t)round_up(K, kOzBK), nbp = (size_t)round_up(nb, kOzBN);
  return kOzS * ((size_t)n + nbp) * Kp * sizeof(__nv_bfloat16) + ((size_t)n + nbp) * sizeof(int) +
         1024;
}

bool ozaki_nn_supported(int K) { return K >= 1 && K <= kOzMaxK; }

cudaError_t launch_ozaki_nn(cudaStream_t st, int n, const double* A, int lda, int K,
                            const double* B, int ldb, int nb, double* C, int ldc, bool subtract,
                            void* work) {
  if (n <= 0 || nb <= 0 || K <= 0) return cudaSuccess;
  if (K > kOzMaxK) return cudaErrorInvalidValue;
  const int Kp = round_up(K, kOzBK), nbp = round_up(nb, kOzBN);
  char* w = static_cast<char*>(work);
  __nv_bfloat16* PA = reinterpret_cast<__nv_bfloat16*>(w);
  __nv_bfloat16* PB = PA + (size_t)kOzS * n * Kp;
  int* EA = reinterpret_cast<int*>(PB + (size_t)kOzS * nbp * Kp);
  int* EB = EA + n;
  oz_row_exp_kernel<<<ceil_div((long long)n * 32, 256) < 16 * kSMs ? ceil_div((long long)n * 32, 256) : 16 * kSMs,
                      256, 0, st>>>(n, A, lda, K, EA); note_launch();
  oz_split_rows_kernel<<<16 * kSMs, 256, 0, st>>>(n, A, lda, K, Kp, EA, PA); note_launch();
  oz_split_cols_kernel<<<ceil_div((long long)nbp * 32, 256), 256, 0, st>>>(K, nb, B, ldb, Kp, nbp, EB,
                                                                            PB); note_launch();
  dim3 grid(ceil_div(n, kOzBM), nbp / kOzBN);
  const size_t smem = sizeof(__nv_bfloat16) * 2 * kOzS * (kOzBM + kOzBN) * kOzRowStride;
  static bool attr_done[2] = {false, false};
  if (!attr_done[subtract ? 1 : 0]) {
    cudaError_t e = subtract ? cudaFuncSetAttribute(oz_gemm_kernel<true>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                             : cudaFuncSetAttribute(oz_gemm_kernel<false>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done[subtract ? 1 : 0] = true;
  }
  if (subtract)
    oz_gemm_kernel<true><<<grid, 256, smem, st>>>(n, nb, Kp, PA, EA, PB, nbp, EB, C, ldc);
  else
    oz_gemm_kernel<false><<<grid, 256, smem, st>>>(n, nb, Kp, PA, EA, PB, nbp, EB, C, ldc);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bchdav
