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
// it holds a leading digit and 32 * 32 otherwise, so for K <= 1170 the float32
// accumulation is exact (1170 * (4096 + 2 * 2048 + 6 * 1024) < 2^24).  The
// eight level sums are combined in float64 in the epilogue.
//
// Gram products A^T B reduce over the N rows, where one exponent per column would tie every
// entry to the column's largest one (a hub vertex of a power-law graph costs the other rows
// their low bits).  There the exponents are per column AND per chunk of kOzChunk = 1024 rows:
// each chunk's level sums are exact in float32 by themselves and are scaled by
// 2^{E_chunk,i + F_chunk,k} as they are folded into float64.
//
// Products: legacy warp-level mma.sync m16n8k16 (bf16 in, f32 accumulate).
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.cuh"

namespace bchdav {

constexpr int kOzS = 8;          // slices
constexpr int kOzBits = 6;       // bits per slice
constexpr int kOzMaxK = 448;     // bound used for the one-shot products (exact up to 1092)
constexpr int kOzBM = 64;        // CTA tile rows
constexpr int kOzBN = 32;        // CTA tile columns
constexpr int kOzBK = 16;        // k step
constexpr int kOzStages = 3;     // cp.async pipeline depth
// shared-memory tile rows are 16 bf16 (two 16-byte halves); half h of row r is stored at
// position h ^ ((r >> 2) & 1), so that the eight rows a fragment load touches fall on
// distinct banks without padding
__device__ __forceinline__ int oz_sw(int r, int half) { return r * 16 + ((half ^ ((r >> 2) & 1)) << 3); }
constexpr int kOzChunk = 1024;   // rows per exponent chunk of a Gram operand (64 k steps of 16)

// Digit planes are stored tiled for the tensor cores.  Element (s, r, k) of the planes of an
// operand with `rows` rows (k the reduction index, padded to a multiple of 16) sits at
//     ((((k / 16) * 8 + s) * 2 + (k / 8) % 2) * rows + r) * 8 + k % 8      (bf16 units),
// so that one 16-wide k step of any run of consecutive rows is, for each slice and each half of
// the step, one contiguous block of 16 bytes per row: the K-major 8 x 16-byte core matrices the
// tcgen05 products read (a 128-row tile: 2 KB per slice and half, fetched by one TMA box for all
// slices), and 16-byte pieces at consecutive addresses for the warp-level kernel's cp.async.
__host__ __device__ __forceinline__ size_t oz_tix(int s, size_t r, int k, size_t rows) {
  return (((((size_t)(k >> 4) * kOzS + s) * 2 + ((k >> 3) & 1)) * rows + r) << 3) + (k & 7);
}

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

// bf16 bit patterns (in the high 16 bits of f[s]) of the balanced base-64 digits of a, most
// significant first: F = round(|a| 2^(48 - E)) = sum_s d_s 64^(7 - s), d_0 in [0, 64],
// d_1..d_7 in [-32, 31], each carrying the sign of a.  The digits come from the two 24-bit
// halves of F with 32-bit integer operations (the low half's four digits leave a carry of 0
// or 1 for the high half).  A digit v (|v| <= 64) becomes a float by adding it to the bit
// pattern of 1.5 * 2^23 and subtracting 1.5 * 2^23 (exact below 2^22), and that float's low 16
// bits are zero, so its high half is the bf16 pattern.
__device__ __forceinline__ void oz_split_bits(double a, int E, uint32_t (&f)[kOzS]) {
  const unsigned long long F = oz_fixed(a, E);
  int lo = (int)(F & 0xFFFFFFull), hi = (int)(F >> 24);
  const int m = (__double2hiint(a) < 0) ? -1 : 0;   // sign of a
  int d[kOzS];
#pragma unroll
  for (int s = kOzS - 1; s >= 4; --s) {
    const int r = ((lo + 32) & 63) - 32;
    d[s] = r;
    lo = (lo - r) >> 6;
  }
  hi += lo;
#pragma unroll
  for (int s = 3; s >= 1; --s) {
    const int r = ((hi + 32) & 63) - 32;
    d[s] = r;
    hi = (hi - r) >> 6;
  }
  d[0] = hi;
#pragma unroll
  for (int s = 0; s < kOzS; ++s) {
    const int v = (d[s] ^ m) - m;
    f[s] = __float_as_uint(__int_as_float(0x4B400000 + v) - 12582912.0f);
  }
}

// two elements' patterns packed as bf16 pairs (first element in the low half)
__device__ __forceinline__ uint32_t oz_pack(uint32_t f0, uint32_t f1) {
  return __byte_perm(f0, f1, 0x7632);
}

__device__ __forceinline__ double oz_pow2(int ex) {
  return (ex > -1022 && ex < 1023) ? __longlong_as_double((long long)(ex + 1023) << 52)
                                   : ldexp(1.0, ex);
}

// Row exponents and slices of A (N x K, K <= kOzMaxK) into tiled planes with `n` rows and Kp
// (zero padded) values of k, in one pass over A: a CTA stages R whole rows in shared memory
// (row-contiguous, coalesced loads; R ~ 4096 / Kp, 16 to 128), takes each row's exponent
// E[i] = max_j (exponent(a_ij) + 1) (0 for a zero row), then thread t splits 8 consecutive k of
// one row and stores one 16-byte piece per slice (consecutive threads: consecutive rows).
constexpr int kOzSRowsMin = 16, kOzSRowsMax = 128;
__host__ __device__ inline int oz_srows(int Kp) {
  const int r = 4096 / (Kp > 0 ? Kp : 1);
  return r < kOzSRowsMin ? kOzSRowsMin : (r > kOzSRowsMax ? kOzSRowsMax : r);
}

__global__ void __launch_bounds__(256) oz_slice_rows_kernel(int n, const double* __restrict__ A,
                                                            int lda, int K, int Kp,
                                                            const double* __restrict__ colscale,
                                                            int slices, int* __restrict__ E,
                                                            __nv_bfloat16* __restrict__ P) {
  extern __shared__ double oz_rtile[];   // R x (Kp + 1)
  __shared__ int s_e[kOzSRowsMax];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int ld = Kp + 1;
  const int R = oz_srows(Kp);
  const int r0 = blockIdx.x * R;
  for (int i = warp; i < R; i += 8) {
    const int r = r0 + i;
    int mx = -100000;
    for (int k = lane; k < Kp; k += 32) {
      double a = (r < n && k < K) ? A[(size_t)r * lda + k] : 0.0;
      if (colscale != nullptr && k < K) a *= colscale[k];   // a power of two: exact
      oz_rtile[i * ld + k] = a;
      mx = max(mx, oz_exp_plus1(a));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      const int e = (mx < -50000) ? 0 : mx;
      s_e[i] = e;
      if (r < n) E[r] = e;
    }
  }
  __syncthreads();
  const int groups = Kp >> 3;
  for (int item = t; item < R * groups; item += 256) {
    const int i = item % R, g = item / R;
    const int r = r0 + i;
    if (r >= n) continue;
    const int e = s_e[i];
    const double* row = oz_rtile + i * ld + 8 * g;
    uint32_t w[kOzS][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      uint32_t f0[kOzS], f1[kOzS];
      oz_split_bits(row[j], e, f0);
      oz_split_bits(row[j + 1], e, f1);
#pragma unroll
      for (int s = 0; s < kOzS; ++s) w[s][j >> 1] = oz_pack(f0[s], f1[s]);
    }
#pragma unroll
    for (int s = 0; s < kOzS; ++s)
      if (s < slices)   // a product that reads only the leading slices needs only those
        *reinterpret_cast<uint4*>(P + oz_tix(s, r, 8 * g, n)) =
            make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
  }
}

static cudaError_t oz_slice_rows_launch(cudaStream_t st, int n, const double* A, int lda, int K,
                                        int Kp, int* E, __nv_bfloat16* P,
                                        const double* colscale = nullptr, int slices = kOzS) {
  if (Kp > kOzMaxK || Kp % 8 != 0) return cudaErrorInvalidValue;
  const int R = oz_srows(Kp);
  const size_t smem = (size_t)R * (Kp + 1) * sizeof(double);
  static const bool attr = [] {
    size_t mx = 0;
    for (int kp = 16; kp <= kOzMaxK; kp += 16)
      mx = std::max(mx, (size_t)oz_srows(kp) * (kp + 1) * sizeof(double));
    return cudaFuncSetAttribute(oz_slice_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mx) == cudaSuccess;
  }();
  if (!attr) return cudaErrorInvalidValue;
  oz_slice_rows_kernel<<<ceil_div(n, R), 256, smem, st>>>(n, A, lda, K, Kp, colscale, slices, E,
                                                          P);
  note_launch();
  return cudaGetLastError();
}

// Column exponents and transposed slices of B (K x nb): planes S x nbp x Kp.
__global__ void oz_split_cols_kernel(int K, int nb, const double* __restrict__ B, int ldb, int Kp,
                                     int nbp, int* __restrict__ F_out, __nv_bfloat16* __restrict__ P) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nbp; c += warps) {
    int m = -100000;
    if (c < nb)
      for (int k = lane; k < K; k += 32) m = max(m, oz_exp_plus1(B[(size_t)k * ldb + c]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int Ec = (m < -50000) ? 0 : m;
    if (lane == 0) F_out[c] = Ec;
    for (int k = lane; k < Kp; k += 32) {
      const double b = (c < nb && k < K) ? B[(size_t)k * ldb + c] : 0.0;
      uint32_t f[kOzS];
      oz_split_bits(b, Ec, f);
#pragma unroll
      for (int s = 0; s < kOzS; ++s)
        P[oz_tix(s, c, k, nbp)] = __ushort_as_bfloat16((unsigned short)(f[s] >> 16));
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

// four 8x8 bf16 matrices from shared memory, one row address per lane (lanes 8i..8i+7 for
// matrix i); lane t receives row t/4, columns 2(t%4), 2(t%4)+1 of each: the mma fragment layout
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* smem_row) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem_row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Slice product.  Rows of the result come from rows a0 .. a0 + M - 1 of the tiled planes PA
// (Ma rows), columns from the tiled planes PB (Np rows).  CTA: 8 warps as 4 (rows) x 2 (cols), warp tile 16 x 16 (one
// m16 tile, two n8 tiles); k steps of 16 double-buffered through shared memory.  blockIdx.z
// takes k steps [z * k_split, (z + 1) * k_split).  The float32 level sums are folded into
// float64 every kOzFlush k steps (1024 values of k, inside the exactness bound) and at the end.
// MODE 0: C = result; 1: C -= result; 2: partial[z] (M x N, row-major) = result.
constexpr int kOzFlush = 64;

// NS: leading digit slices used (8: float64-accurate; fewer: a truncated product whose
// operands keep 6 NS bits, for the first DGKS pass that the second one corrects)
template <int MODE, int NS>
__global__ void __launch_bounds__(256, 2) oz_gemm_kernel(int M, int Ma, int a0, int N, int Kp,
                                                      int k_split,
                                                      const __nv_bfloat16* __restrict__ PA,
                                                      const int* __restrict__ EA,
                                                      const __nv_bfloat16* __restrict__ PB, int Np,
                                                      const int* __restrict__ EB,
                                                      double* __restrict__ C, int ldc) {
  extern __shared__ __align__(16) unsigned char oz_smem[];
  // sA[stage][s][swizzled row-major 64 x 16], sB likewise (32 x 16), then 8 float64 per
  // thread (88 KB of dynamic shared memory: two CTAs per SM)
  auto sA = reinterpret_cast<__nv_bfloat16(*)[kOzS][kOzBM * 16]>(oz_smem);
  auto sB = reinterpret_cast<__nv_bfloat16(*)[kOzS][kOzBN * 16]>(
      oz_smem + sizeof(__nv_bfloat16) * kOzStages * kOzS * kOzBM * 16);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int wm = warp & 3, wn = warp >> 2;
  // MODE 0/1 (A's rows are the output rows, B small): a flat grid with the column tiles of a row
  // tile adjacent, so that they find A's tile in L2 (one DRAM pass over A); MODE 2: (M tile,
  // N tile, k split)
  const int nct = Np / kOzBN;
  const int r0 = MODE == 2 ? blockIdx.x * kOzBM : (int)(blockIdx.x / nct) * kOzBM;
  const int c0 = MODE == 2 ? blockIdx.y * kOzBN : (int)(blockIdx.x % nct) * kOzBN;
  const int g = lane >> 2, tig = lane & 3;
  const int nk_all = Kp / kOzBK;
  const int kt0 = blockIdx.z * k_split;
  const int kt1 = min(nk_all, kt0 + k_split);

  auto load_stage = [&](int buf, int k0) {
    for (int q = t; q < NS * kOzBM * 2; q += 256) {
      const int s = q / (kOzBM * 2), rem = q - s * kOzBM * 2, row = rem >> 1, half = rem & 1;
      const int gr = r0 + row;
      __nv_bfloat16* dst = &sA[buf][s][oz_sw(row, half)];
      if (gr < M) cp_async16(dst, PA + oz_tix(s, (size_t)a0 + gr, k0 + half * 8, Ma));
      else *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
    }
    for (int q = t; q < NS * kOzBN * 2; q += 256) {
      const int s = q / (kOzBN * 2), rem = q - s * kOzBN * 2, row = rem >> 1, half = rem & 1;
      const int gc = c0 + row;
      __nv_bfloat16* dst = &sB[buf][s][oz_sw(row, half)];
      if (gc < Np) cp_async16(dst, PB + oz_tix(s, gc, k0 + half * 8, Np));
      else *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
    }
    cp_async_commit();
  };

  float acc[NS][2][4];
  // float64 partial sums live in shared memory (touched only at flushes), 8 per thread
  double* dacc = reinterpret_cast<double*>(
      oz_smem + sizeof(__nv_bfloat16) * kOzStages * kOzS * (kOzBM + kOzBN) * 16) + t * 8;
#pragma unroll
  for (int e = 0; e < 8; ++e) dacc[e] = 0.0;
  auto zero_acc = [&]() {
#pragma unroll
    for (int L = 0; L < NS; ++L)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[L][j][e] = 0.f;
  };
  // MODE 2: chunk exponents, the k steps folded last lie in chunk `ch`
  // The level sums are integers (exact in float32), so they are combined exactly in 64-bit
  // integers and converted to float64 once: hi = sum_{L < H} acc_L 2^(6 (H - 1 - L)) and
  // lo = sum_{L >= H} acc_L 2^(6 (NS - 1 - L)), H = NS / 2, each below 2^42 for the 1024-row
  // pieces of a Gram product; value = (hi 2^(6 (NS - H)) + lo) 2^(-6 (NS + 1)).
  auto flush = [&](int ch) {
    constexpr int kH = NS / 2;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        long long hi = 0, lo = 0;
#pragma unroll
        for (int L = 0; L < NS; ++L) {
          const long long q = (long long)__float2int_rn(acc[L][j][e]);
          if (L < kH) hi += q * (1LL << (kOzBits * (kH - 1 - L)));
          else lo += q * (1LL << (kOzBits * (NS - 1 - L)));
        }
        double v = fma((double)hi, (double)(1LL << (kOzBits * (NS - kH))), (double)lo) *
                   __longlong_as_double((long long)(1023 - kOzBits * (NS + 1)) << 52);
        if (MODE == 2) {
          const int row = r0 + wm * 16 + g + (e >> 1) * 8;
          const int col = c0 + wn * 16 + j * 8 + tig * 2 + (e & 1);
          v = (row < M && col < N)
                  ? v * oz_pow2(EA[(size_t)ch * Ma + row] + EB[(size_t)ch * Np + col])
                  : 0.0;
        }
        dacc[j * 4 + e] += v;
      }
    zero_acc();
  };
  zero_acc();

  const int nst = kt1 - kt0;
  if (nst > 0) load_stage(0, kt0 * kOzBK);
  if (nst > 1) load_stage(1, (kt0 + 1) * kOzBK);
  for (int kt = kt0; kt < kt1; ++kt) {
    const int i = kt - kt0, buf = i % kOzStages;
    // stage i has landed once at most one later group is pending
    if (i + 1 < nst) cp_async_wait<1>();
    else cp_async_wait0();
    __syncthreads();
    if (i + 2 < nst) load_stage((i + 2) % kOzStages, (kt + 2) * kOzBK);
    // fragments by ldmatrix: lane l addresses row (l & 7) of matrix l >> 3
    const int mi = lane >> 3, rr = lane & 7;
    uint32_t bf[NS][2][2];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      // matrices: (n-tile 0, k half 0), (0, 1), (1, 0), (1, 1)
      uint32_t q[4];
      ldsm_x4(q, &sB[buf][s][oz_sw(wn * 16 + (mi >> 1) * 8 + rr, mi & 1)]);
      bf[s][0][0] = q[0];
      bf[s][0][1] = q[1];
      bf[s][1][0] = q[2];
      bf[s][1][1] = q[3];
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      // matrices: (rows 0-7, k half 0), (rows 8-15, 0), (rows 0-7, 1), (rows 8-15, 1)
      uint32_t af[4];
      ldsm_x4(af, &sA[buf][s][oz_sw(wm * 16 + (mi & 1) * 8 + rr, mi >> 1)]);
#pragma unroll
      for (int tt = 0; tt < NS; ++tt) {
        if (s + tt < NS) {   // levels s + tt + 2 <= NS + 1
          oz_mma(acc[s + tt][0], af, bf[tt][0]);
          oz_mma(acc[s + tt][1], af, bf[tt][1]);
        }
      }
    }
    if (((kt - kt0 + 1) % kOzFlush) == 0) flush(kt / kOzFlush);
  }
  flush(kt1 > kt0 ? (kt1 - 1) / kOzFlush : 0);
  // epilogue: scale by 2^(E_row + F_col)
#pragma unroll
  for (int j = 0; j < 2; ++j) {
#pragma unroll
    for (int hrow = 0; hrow < 2; ++hrow) {
      const int row = r0 + wm * 16 + g + hrow * 8;
      if (row >= M) continue;
      const int Er = MODE == 2 ? 0 : EA[row];
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int col = c0 + wn * 16 + j * 8 + tig * 2 + cc;
        if (col >= N) continue;
        const double scale = MODE == 2 ? 1.0 : oz_pow2(Er + EB[col]);
        const double v = dacc[j * 4 + hrow * 2 + cc] * scale;
        if (MODE == 0) C[(size_t)row * ldc + col] = v;
        else if (MODE == 1) C[(size_t)row * ldc + col] -= v;
        else C[(size_t)blockIdx.z * M * N + (size_t)row * N + col] = v;
      }
    }
  }
}

template <int MODE, int NS = kOzS>
static cudaError_t oz_launch_gemm(cudaStream_t st, dim3 grid, int M, int Ma, int a0, int N, int Kp,
                                  int k_split, const __nv_bfloat16* PA, const int* EA,
                                  const __nv_bfloat16* PB, int Np, const int* EB, double* C,
                                  int ldc) {
  const size_t smem = sizeof(__nv_bfloat16) * kOzStages * kOzS * (kOzBM + kOzBN) * 16 +
                      256 * 8 * sizeof(double);
  // set once per process (thread-safe static initialisation)
  static const cudaError_t attr = cudaFuncSetAttribute(
      oz_gemm_kernel<MODE, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (attr != cudaSuccess) return attr;
  oz_gemm_kernel<MODE, NS><<<grid, 256, smem, st>>>(M, Ma, a0, N, Kp, k_split, PA, EA, PB, Np, EB,
                                                    C, ldc);
  note_launch();
  return cudaGetLastError();
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
  cudaError_t es = oz_slice_rows_launch(st, n, A, lda, K, Kp, EA, PA);
  if (es != cudaSuccess) return es;
  oz_split_cols_kernel<<<ceil_div((long long)nbp * 32, 256), 256, 0, st>>>(K, nb, B, ldb, Kp, nbp, EB,
                                                                            PB); note_launch();
  dim3 grid((unsigned)((long long)ceil_div(n, kOzBM) * (nbp / kOzBN)), 1, 1);
  const int ks = Kp / kOzBK;
  if (subtract) return oz_launch_gemm<1>(st, grid, n, n, 0, nb, Kp, ks, PA, EA, PB, nbp, EB, C, ldc);
  return oz_launch_gemm<0>(st, grid, n, n, 0, nb, Kp, ks, PA, EA, PB, nbp, EB, C, ldc);
}

// ---------------- Gram products A^T B (reduction over the N rows) ----------------
int oz_chunks(int Np) { return ceil_div(Np, kOzChunk); }

size_t ozaki_tn_work_bytes(int n, int ka, int kb) {
  const size_t Np = (size_t)round_up(n, kOzBK);
  const size_t kap = (size_t)round_up(ka, kOzBM), kbp = (size_t)round_up(kb, kOzBN);
  const size_t splits = 4 * kSMs;
  return kOzS * (kap + kbp) * Np * sizeof(__nv_bfloat16) +
         (kap + kbp) * (size_t)oz_chunks((int)Np) * sizeof(int) +
         splits * (size_t)ka * kb * sizeof(double) + 4096;
}

cudaError_t launch_ozaki_tn(cudaStream_t st, int n, const double* A, int lda, int ka,
                            const double* B, int ldb, int kb, double* out, void* work,
                            int* tc_err) {
  if (n <= 0 || ka <= 0 || kb <= 0) return cudaSuccess;
  const int Np = round_up(n, kOzBK);
  const int kap = round_up(ka, kOzBM), kbp = round_up(kb, kOzBN);
  char* w = static_cast<char*>(work);
  __nv_bfloat16* PA = reinterpret_cast<__nv_bfloat16*>(w);
  __nv_bfloat16* PB = PA + (size_t)kOzS * kap * Np;
  const int nch = oz_chunks(Np);
  int* EA = reinterpret_cast<int*>(PB + (size_t)kOzS * kbp * Np);
  int* EB = EA + (size_t)kap * nch;
  int* Eend = EB + (size_t)kbp * nch;
  double* partial = reinterpret_cast<double*>(
      reinterpret_cast<char*>(Eend) + (256 - (reinterpret_cast<uintptr_t>(Eend) & 255)));
  cudaError_t e0 = oz_slice_cols_t(st, n, A, lda, ka, Np, kap, 0, PA, EA);
  if (e0 != cudaSuccess) return e0;
  e0 = oz_slice_cols_t(st, n, B, ldb, kb, Np, kbp, 0, PB, EB);
  if (e0 != cudaSuccess) return e0;
  if (tc_err != nullptr)   // tcgen05 products with tensor-memory level sums (tc05.cu)
    return launch_tc_gram(st, Np, PA, EA, kap, 0, ka, PB, EB, kbp, kb, out, partial, kOzS, tc_err);
  // split the reduction so that the grid covers the GPU about twice
  const int tiles = (kap / kOzBM) * (kbp / kOzBN);
  const int nk = Np / kOzBK;
  int nsplit = std::max(1, std::min(4 * kSMs, (2 * kSMs + tiles - 1) / tiles));
  // splits start on chunk boundaries (the chunk exponents apply per fold)
  const int k_split = round_up(ceil_div(nk, nsplit), kOzFlush);
  nsplit = ceil_div(nk, k_split);
  dim3 grid(kap / kOzBM, kbp / kOzBN, nsplit);
  cudaError_t e =
      oz_launch_gemm<2>(st, grid, ka, kap, 0, kb, Np, k_split, PA, EA, PB, kbp, EB, partial, kb);
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(st, partial, nsplit, ka * kb, out, 1.0);
}


// ---------------- building blocks for cached slices ----------------
size_t oz_planes_bytes(size_t rows, size_t kp) { return kOzS * rows * kp * sizeof(__nv_bfloat16); }
int oz_pad_k(int k) { return round_up(k, kOzBK); }
int oz_pad_rows(int m) { return round_up(m, kOzBM); }
int oz_pad_cols(int n) { return round_up(n, kOzBN); }

// Row slices of A (n x K) into planes S x n x Kp with exponents E[n].
cudaError_t oz_slice_rows(cudaStream_t st, int n, const double* A, int lda, int K, int Kp,
                          void* planes, int* E, const double* colscale, int slices) {
  if (slices < 1 || slices > kOzS) return cudaErrorInvalidValue;
  return oz_slice_rows_launch(st, n, A, lda, K, Kp, E, static_cast<__nv_bfloat16*>(planes),
                              colscale, slices);
}

// Transposed column slices: columns [0, w) of X (N x w) become rows [c_off, c_off + w) of the
// tiled planes with `cap` rows and Np values of k (the N rows of X, zero padded), with chunk
// exponents E[ch * cap + c_off + c] = max over the rows of chunk ch of (exponent(x_rc) + 1) (0
// for a chunk column without nonzeros), in one pass over X: a CTA stages one chunk (kOzChunk
// rows) of 8 columns in shared memory, takes the 8 exponents (one warp per column), then
// thread t splits 8 consecutive rows of one column and stores one 16-byte piece per slice
// (consecutive threads: consecutive columns, 128 contiguous bytes per slice).  Rows of the
// planes outside [c_off, c_off + w) are untouched.
constexpr int kOzTCols = 8;
constexpr int kOzTLd = kOzChunk + 2;   // doubles per staged column

__global__ void __launch_bounds__(256) oz_slice_cols_kernel(
    int n, const double* __restrict__ X, int ldx, int w, int Np, int cap, int c_off,
    int* __restrict__ E, __nv_bfloat16* __restrict__ P) {
  extern __shared__ double oz_ctile[];   // [kOzTCols][kOzTLd]
  __shared__ int s_e[kOzTCols];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int ch = blockIdx.x, c0 = blockIdx.y * kOzTCols;
  const int r0 = ch * kOzChunk;
  const int rows = min(kOzChunk, Np - r0);   // a multiple of 8
  for (int idx = t; idx < kOzChunk * kOzTCols; idx += 256) {
    const int rl = idx / kOzTCols, cl = idx % kOzTCols;
    const int r = r0 + rl, c = c0 + cl;
    oz_ctile[cl * kOzTLd + rl] = (r < n && c < w) ? X[(size_t)r * ldx + c] : 0.0;
  }
  __syncthreads();
  {
    const int cl = warp;   // 8 warps, 8 columns
    int mx = -100000;
    for (int rl = lane; rl < rows; rl += 32) mx = max(mx, oz_exp_plus1(oz_ctile[cl * kOzTLd + rl]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      const int e = (mx < -50000) ? 0 : mx;
      s_e[cl] = e;
      if (c0 + cl < w) E[(size_t)ch * cap + c_off + c0 + cl] = e;
    }
  }
  __syncthreads();
  const int groups = rows >> 3;
  for (int item = t; item < kOzTCols * groups; item += 256) {
    const int cl = item % kOzTCols, g = item / kOzTCols;
    const int c = c0 + cl;
    if (c >= w) continue;
    const int e = s_e[cl];
    const double* col = oz_ctile + cl * kOzTLd + 8 * g;
    uint32_t wd[kOzS][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      uint32_t f0[kOzS], f1[kOzS];
      oz_split_bits(col[j], e, f0);
      oz_split_bits(col[j + 1], e, f1);
#pragma unroll
      for (int s = 0; s < kOzS; ++s) wd[s][j >> 1] = oz_pack(f0[s], f1[s]);
    }
#pragma unroll
    for (int s = 0; s < kOzS; ++s)
      *reinterpret_cast<uint4*>(P + oz_tix(s, (size_t)c_off + c, r0 + 8 * g, cap)) =
          make_uint4(wd[s][0], wd[s][1], wd[s][2], wd[s][3]);
  }
}

cudaError_t oz_slice_cols_t(cudaStream_t st, int n, const double* A, int lda, int w, int Np, int cap,
                            int c_off, void* planes, int* E) {
  if (w <= 0) return cudaSuccess;
  if (Np % 8 != 0) return cudaErrorInvalidValue;
  const size_t smem = (size_t)kOzTCols * kOzTLd * sizeof(double);
  static const bool attr = [smem] {
    return cudaFuncSetAttribute(oz_slice_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem) == cudaSuccess;
  }();
  if (!attr) return cudaErrorInvalidValue;
  dim3 g(oz_chunks(Np), ceil_div(w, kOzTCols));
  oz_slice_cols_kernel<<<g, 256, smem, st>>>(n, A, lda, w, Np, cap, c_off, E,
                                             static_cast<__nv_bfloat16*>(planes));
  note_launch();
  return cudaGetLastError();
}

// out (ka x kb) = A^T B from transposed planes: rows [a0, a0 + ka) of PA (S x capA x Np,
// chunk exponents EA, stride capA) and rows [0, kb) of PB (S x capB x Np, chunk exponents EB,
// stride capB; capB >= round_up(kb, 32)).
cudaError_t oz_gram_from_planes(cudaStream_t st, int Np, const void* PA, const int* EA, int capA,
                                int a0, int ka, const void* PB, const int* EB, int capB, int kb,
                                double* out, double* partial, int slices) {
  if (ka <= 0 || kb <= 0) return cudaSuccess;
  const __nv_bfloat16* pa = static_cast<const __nv_bfloat16*>(PA);
  const __nv_bfloat16* pb = static_cast<const __nv_bfloat16*>(PB);
  const int mt = ceil_div(ka, kOzBM), nt = ceil_div(kb, kOzBN);
  const int tiles = mt * nt;
  const int nk = Np / kOzBK;
  int nsplit = std::max(1, std::min(4 * kSMs, (2 * kSMs + tiles - 1) / tiles));
  const int k_split = round_up(ceil_div(nk, nsplit), kOzFlush);   // chunk-aligned splits
  nsplit = ceil_div(nk, k_split);
  dim3 grid(mt, nt, nsplit);
  // rows a0 .. a0 + ka - 1 of A's planes (capA rows)
  cudaError_t e;
  if (slices == 4)
    e = oz_launch_gemm<2, 4>(st, grid, ka, capA, a0, kb, Np, k_split, pa, EA + a0, pb, capB, EB,
                             partial, kb);
  else if (slices == 6)
    e = oz_launch_gemm<2, 6>(st, grid, ka, capA, a0, kb, Np, k_split, pa, EA + a0, pb, capB, EB,
                             partial, kb);
  else if (slices == kOzS)
    e = oz_launch_gemm<2>(st, grid, ka, capA, a0, kb, Np, k_split, pa, EA + a0, pb, capB, EB,
                          partial, kb);
  else
    return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(st, partial, nsplit, ka * kb, out, 1.0);
}

// C (n x nb) = / -= A B from row planes of A (S x n x Kp, exponents EA) and a small B (K x nb).
cudaError_t oz_nn_from_planes(cudaStream_t st, int n, int K, int Kp, const void* PA, const int* EA,
                              const double* B, int ldb, int nb, double* C, int ldc, bool subtract,
                              void* bwork, int slices) {
  if (n <= 0 || nb <= 0 || K <= 0) return cudaSuccess;
  if (K > kOzMaxK) return cudaErrorInvalidValue;
  const int nbp = round_up(nb, kOzBN);
  __nv_bfloat16* PB = static_cast<__nv_bfloat16*>(bwork);
  int* EB = reinterpret_cast<int*>(PB + (size_t)kOzS * nbp * Kp);
  oz_split_cols_kernel<<<ceil_div((long long)nbp * 32, 256), 256, 0, st>>>(K, nb, B, ldb, Kp, nbp, EB,
                                                                            PB); note_launch();
  dim3 grid((unsigned)((long long)ceil_div(n, kOzBM) * (nbp / kOzBN)), 1, 1);
  const __nv_bfloat16* pa = static_cast<const __nv_bfloat16*>(PA);
  // the subtraction X -= V C always uses every slice (its error must stay inside span(V));
  // the product C = A B may use 6 (operands to 36 bits)
  if (subtract) {
    if (slices != kOzS) return cudaErrorInvalidValue;
    return oz_launch_gemm<1>(st, grid, n, n, 0, nb, Kp, Kp / kOzBK, pa, EA, PB, nbp, EB, C, ldc);
  }
  if (slices == 6)
    return oz_launch_gemm<0, 6>(st, grid, n, n, 0, nb, Kp, Kp / kOzBK, pa, EA, PB, nbp, EB, C, ldc);
  if (slices != kOzS) return cudaErrorInvalidValue;
  return oz_launch_gemm<0>(st, grid, n, n, 0, nb, Kp, Kp / kOzBK, pa, EA, PB, nbp, EB, C, ldc);
}

cudaError_t oz_nn_from_planes_tc(cudaStream_t st, int n, int K, int Kp, const void* PA,
                                 const int* EA, const double* B, int ldb, int nb, double* C,
                                 int ldc, bool subtract, void* bwork, int slices, int* err) {
  if (n <= 0 || nb <= 0 || K <= 0) return cudaSuccess;
  if (K > kOzMaxK) return cudaErrorInvalidValue;
  const int nbp = nb <= 32 ? 32 : round_up(nb, 64);
  __nv_bfloat16* PB = static_cast<__nv_bfloat16*>(bwork);
  int* EB = reinterpret_cast<int*>(PB + (size_t)kOzS * nbp * Kp);
  oz_split_cols_kernel<<<ceil_div((long long)nbp * 32, 256), 256, 0, st>>>(K, nb, B, ldb, Kp, nbp, EB,
                                                                            PB); note_launch();
  return launch_tc_slice_nn(st, n, nb, Kp, PA, EA, PB, nbp, EB, C, ldc, subtract, slices, err);
}

size_t oz_bwork_bytes(int K, int nb) {
  const size_t nbp = (size_t)round_up(nb, 64);   // covers both slice-product kernels' padding
  return kOzS * nbp * round_up(K, kOzBK) * sizeof(__nv_bfloat16) + nbp * sizeof(int) + 256;
}

}  // namespace bchdav
