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
#include <algorithm>

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

// The row's nonzeros in batches of four: the four colidx/val loads are independent, then the
// four gathers.  A batch past the row's end loads the row's own X row (in bounds, read again
// by the epilogue) and skips its multiply-add, so a row of length L costs ceil(L / 4)
// dependent load rounds and the sum runs in the order of the nonzeros (k ascending).
template <typename T, int VW>
__device__ __forceinline__ void row_product(const int* __restrict__ colidx, const T* __restrict__ val,
                                            const T* __restrict__ X, int ldx, int c0, int row,
                                            int start, int end, T (&acc)[VW]) {
  for (int k = start; k < end; k += 4) {
    int j[4];
    T a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool ok = k + u < end;
      j[u] = ok ? __ldg(colidx + k + u) : row;
      a[u] = ok ? __ldg(val + k + u) : T(0);
    }
    T x[4][VW];
#pragma unroll
    for (int u = 0; u < 4; ++u) ldv<T, VW>(X + (size_t)j[u] * ldx + c0, x[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (k + u < end)
#pragma unroll
        for (int i = 0; i < VW; ++i) acc[i] = fma(a[u], x[u][i], acc[i]);
  }
}

// ---------------- long rows: fixed-size segments, reduced in a fixed order ----------------
// A row with more than kLongRow nonzeros would keep one row group busy for its whole length
// (power-law graphs have rows of 10^5 entries), so such rows are cut into segments of kLongRow
// nonzeros.  One CTA computes each segment's partial product into pseg (segment-major, b
// values); the row kernel then adds a long row's segments in segment order.  Both sums run in
// a fixed order: results do not depend on scheduling.
__global__ void long_count_segments_kernel(int n, const int* __restrict__ rowptr,
                                           int* __restrict__ cnt) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int len = rowptr[r + 1] - rowptr[r];
    cnt[r] = len > kLongRow ? (len + kLongRow - 1) / kLongRow : 0;
  }
}

__global__ void long_fill_rows_kernel(int n, const long long* __restrict__ seg_off,
                                      int* __restrict__ seg_row) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    for (long long s = seg_off[r]; s < seg_off[r + 1]; ++s) seg_row[s] = r;
}

cudaError_t build_spmm_long(cudaStream_t st, int n, const int* rowptr, int* cnt_work,
                            long long* seg_off, long long* tile_sums, int* seg_row,
                            long long seg_cap, long long* host_total, long long* n_seg) {
  *n_seg = 0;
  if (n <= 0) return cudaSuccess;
  const int grid = std::min(ceil_div(n, 256), 16 * kSMs);
  long_count_segments_kernel<<<grid, 256, 0, st>>>(n, rowptr, cnt_work); note_launch();
  cudaError_t e = exclusive_scan(st, n, cnt_work, 0, seg_off, tile_sums);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(host_total, seg_off + n, sizeof(long long), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  if (*host_total > seg_cap) return cudaErrorInvalidValue;
  *n_seg = *host_total;
  if (*n_seg > 0) {
    long_fill_rows_kernel<<<grid, 256, 0, st>>>(n, seg_off, seg_row); note_launch();
  }
  return cudaGetLastError();
}

long long spmm_long_seg_cap(long long nnz) { return 2 * (nnz / kLongRow) + 1; }

// One CTA per segment: the segment's colidx/val are staged in shared memory by all threads
// (independent loads), then G row groups of tpr threads each gather every G-th entry; the
// group sums are added in group order.
template <typename T, int VW>
__global__ void __launch_bounds__(256) spmm_long_seg_kernel(
    const int* __restrict__ rowptr, const int* __restrict__ colidx, const T* __restrict__ val,
    const T* __restrict__ X, int ldx, int b, int tpr, const long long* __restrict__ seg_off,
    const int* __restrict__ seg_row, T* __restrict__ pseg, int ldp) {
  __shared__ int s_col[kLongRow];
  __shared__ T s_val[kLongRow];
  __shared__ T s_red[256 * VW];
  const long long s = blockIdx.x;
  const int row = seg_row[s];
  const long long q0 = rowptr[row] + (s - seg_off[row]) * (long long)kLongRow;
  const int cnt = (int)min((long long)kLongRow, (long long)rowptr[row + 1] - q0);
  for (int e = threadIdx.x; e < cnt; e += 256) {
    s_col[e] = colidx[q0 + e];
    s_val[e] = val[q0 + e];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gpw = 32 / tpr, g_lane = lane / tpr, li = lane - g_lane * tpr;
  const int G = 8 * gpw, g = warp * gpw + g_lane;
  T acc[VW];
#pragma unroll
  for (int i = 0; i < VW; ++i) acc[i] = T(0);
  const int c0 = li * VW;
  if (g_lane < gpw && c0 < b) {
    int e = g;
    for (; e + 3 * G < cnt; e += 4 * G) {
      T x0[VW], x1[VW], x2[VW], x3[VW];
      ldv<T, VW>(X + (size_t)s_col[e] * ldx + c0, x0);
      ldv<T, VW>(X + (size_t)s_col[e + G] * ldx + c0, x1);
      ldv<T, VW>(X + (size_t)s_col[e + 2 * G] * ldx + c0, x2);
      ldv<T, VW>(X + (size_t)s_col[e + 3 * G] * ldx + c0, x3);
      const T a0 = s_val[e], a1 = s_val[e + G], a2 = s_val[e + 2 * G], a3 = s_val[e + 3 * G];
#pragma unroll
      for (int i = 0; i < VW; ++i) {
        acc[i] = fma(a0, x0[i], acc[i]);
        acc[i] = fma(a1, x1[i], acc[i]);
        acc[i] = fma(a2, x2[i], acc[i]);
        acc[i] = fma(a3, x3[i], acc[i]);
      }
    }
    for (; e < cnt; e += G) {
      T x[VW];
      ldv<T, VW>(X + (size_t)s_col[e] * ldx + c0, x);
#pragma unroll
      for (int i = 0; i < VW; ++i) acc[i] = fma(s_val[e], x[i], acc[i]);
    }
  }
  // s_red[g][column]: G groups x b columns (G * b <= 256 * VW)
  if (g_lane < gpw && c0 < b) {
#pragma unroll
    for (int i = 0; i < VW; ++i)
      if (c0 + i < b) s_red[g * b + c0 + i] = acc[i];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < b; c += 256) {
    T t = T(0);
    for (int q = 0; q < G; ++q) t += s_red[q * b + c];
    pseg[s * ldp + c] = t;
  }
}

// ---------------- row kernel ----------------
// A group of tpr consecutive threads owns one row (groups may straddle warps); rpb rows per
// CTA.  Rows longer than kLongRow read their segment sums instead of walking their nonzeros.
template <typename T, int VW>
__global__ void __launch_bounds__(512) spmm_axpby_kernel(
    int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
    const T* __restrict__ val, const T* __restrict__ X, int ldx, int b, T* __restrict__ Y, int ldy,
    const T* __restrict__ Z, int ldz, T alpha, T beta, T gamma, const T* __restrict__ R, int ldr,
    const T* __restrict__ delta, int tpr, int rpb, const long long* __restrict__ seg_off,
    const T* __restrict__ pseg) {
  const int t = threadIdx.x;
  const int rl = t / tpr;
  if (rl >= rpb) return;
  const int row = blockIdx.x * rpb + rl;
  if (row >= n) return;
  const int c0 = (t - rl * tpr) * VW;
  if (c0 >= b) return;   // VW == 1 only: b need not fill the group
  T acc[VW];
#pragma unroll
  for (int i = 0; i < VW; ++i) acc[i] = T(0);
  const int p0 = __ldg(rowptr + row), p1 = __ldg(rowptr + row + 1);
  if (seg_off != nullptr && p1 - p0 > kLongRow) {
    for (long long s = seg_off[row]; s < seg_off[row + 1]; ++s)
#pragma unroll
      for (int i = 0; i < VW; ++i) acc[i] += pseg[s * b + c0 + i];
  } else {
    row_product<T, VW>(colidx, val, X, ldx, c0, row, p0, p1, acc);
  }
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

template <typename T, int VW>
static cudaError_t spmm_rows_launch(cudaStream_t st, int n, const int* rowptr, const int* colidx,
                                    const T* val, const T* X, int ldx, int b, T* Y, int ldy,
                                    const T* Z, int ldz, T alpha, T beta, T gamma, const T* R,
                                    int ldr, const T* delta, int tpr, const SpmmLong* lg,
                                    int threads) {
  const long long* seg_off = nullptr;
  const T* pseg = nullptr;
  if (lg != nullptr && lg->n_seg > 0) {
    if (lg->n_seg > 0x7fffffffLL) return cudaErrorInvalidValue;
    T* ps = static_cast<T*>(lg->pseg);
    if (VW == 1) {
      // one lane per column: at most 32 columns per pass
      for (int c0 = 0; c0 < b; c0 += 32) {
        const int w = std::min(32, b - c0);
        spmm_long_seg_kernel<T, 1><<<(unsigned)lg->n_seg, 256, 0, st>>>(
            rowptr, colidx, val, X + c0, ldx, w, w, lg->seg_off, lg->seg_row, ps + c0, b);
        note_launch();
      }
    } else {
      spmm_long_seg_kernel<T, VW><<<(unsigned)lg->n_seg, 256, 0, st>>>(
          rowptr, colidx, val, X, ldx, b, tpr, lg->seg_off, lg->seg_row, ps, b); note_launch();
    }
    seg_off = lg->seg_off;
    pseg = ps;
  }
  // rows per CTA from the block size (64..512 threads; the caller's schedule, default 256)
  const int bs = threads == 64 || threads == 128 || threads == 512 ? threads : 256;
  const int rpb = std::max(1, bs / tpr);
  const int grid = ceil_div(n, rpb);
  spmm_axpby_kernel<T, VW><<<grid, rpb * tpr, 0, st>>>(n, rowptr, colidx, val, X, ldx, b, Y, ldy,
                                                       Z, ldz, alpha, beta, gamma, R, ldr, delta,
                                                       tpr, rpb, seg_off, pseg); note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spmm_axpby(cudaStream_t st, int n, const int* rowptr, const int* colidx,
                              const T* val, const T* X, int ldx, int b, T* Y, int ldy,
                              const T* Z, int ldz, T alpha, T beta, T gamma, const T* R, int ldr,
                              const T* delta, const SpmmLong* lg, int threads) {
  if (n <= 0 || b <= 0) return cudaSuccess;
  int vw = pick_vw<T>(b, X, ldx, Y, ldy, Z, ldz);
  if (R != nullptr && vw > 1 && (((uintptr_t)R % (vw * sizeof(T))) != 0 || ldr % vw != 0)) vw = 1;
  const int tpr = (b + vw - 1) / vw;
  if (tpr > 256 || (vw > 1 && tpr > 32)) return cudaErrorInvalidValue;
  if (vw == 1)
    return spmm_rows_launch<T, 1>(st, n, rowptr, colidx, val, X, ldx, b, Y, ldy, Z, ldz, alpha,
                                  beta, gamma, R, ldr, delta, tpr, lg, threads);
  if (vw == 2)
    return spmm_rows_launch<T, 2>(st, n, rowptr, colidx, val, X, ldx, b, Y, ldy, Z, ldz, alpha,
                                  beta, gamma, R, ldr, delta, tpr, lg, threads);
  if constexpr (sizeof(T) == 4)
    return spmm_rows_launch<T, 4>(st, n, rowptr, colidx, val, X, ldx, b, Y, ldy, Z, ldz, alpha,
                                  beta, gamma, R, ldr, delta, tpr, lg, threads);
  return cudaErrorInvalidValue;
}

template cudaError_t launch_spmm_axpby<double>(cudaStream_t, int, const int*, const int*,
                                               const double*, const double*, int, int, double*,
                                               int, const double*, int, double, double, double,
                                               const double*, int, const double*,
                                               const SpmmLong*, int);
template cudaError_t launch_spmm_axpby<float>(cudaStream_t, int, const int*, const int*,
                                              const float*, const float*, int, int, float*, int,
                                              const float*, int, float, float, float, const float*,
                                              int, const float*, const SpmmLong*, int);

// ---------------- double-float products (mixed path, Steps 7 and 12) ----------------
// y = A x with A's values and x as unevaluated sums of two floats (hi + lo, ~48 significant
// bits), accumulated in the same form: an exact product error by FMA (two-product) and an
// error-free two-sum per term, about ten float32 operations where float64 takes one FMA.
// GB300's float32 pipe is 64 times wider than its float64 pipe, so the product becomes bound by
// its gathers (the same bytes as float64) instead of float64 arithmetic.  Relative error per
// output about 2^-46 of sum |a_ij x_j|.  The block x is first split into hi/lo floats,
// interleaved per four columns ([4 hi][4 lo], 32 bytes per column group), so that one thread's
// gather is one 32-byte sector.
// x = h + l (l exact up to its float rounding, |l| <= ulp(h) / 2), from the bit pattern with
// integer operations and one int -> float conversion: float64 conversions would run on the
// narrow float64 pipe.  |x| outside [2^-60, 2^61) takes the float64 conversions.
__device__ __forceinline__ void dd_split(double x, float& h, float& l) {
  const long long bits = __double_as_longlong(x);
  const int ef = (int)((bits >> 52) & 0x7FF);
  if (ef < 1023 - 60 || ef > 1023 + 60) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
    return;
  }
  const unsigned neg = (unsigned)((unsigned long long)bits >> 63) << 31;
  const long long m = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);   // |x| = m 2^(ef - 1075)
  long long mh = (m + (1LL << 28)) >> 29;                           // leading 24 bits, rounded
  const int r = (int)(m - (mh << 29));                              // |r| <= 2^28
  int eh = ef - 1023;
  if (mh == (1LL << 24)) {
    mh >>= 1;
    ++eh;
  }
  h = __uint_as_float(neg | ((unsigned)(eh + 127) << 23) | ((unsigned)mh & 0x7FFFFFu));
  const float fr = __int2float_rn(r);   // r 2^(ef - 1075): shift the exponent field
  l = (r == 0) ? 0.f : __uint_as_float((__float_as_uint(fr) + ((unsigned)(ef - 1075) << 23)) ^ neg);
}

__global__ void split_dd_kernel(int n, int b, const double* __restrict__ X, int ldx,
                                float* __restrict__ XD) {
  const int g4 = b >> 2;
  const long long total = (long long)n * g4;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(i / g4), g = (int)(i - (long long)row * g4);
    const double* x = X + (size_t)row * ldx + 4 * g;
    float h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) dd_split(x[j], h[j], l[j]);
    float4* o = reinterpret_cast<float4*>(XD + ((size_t)row * g4 + g) * 8);
    o[0] = make_float4(h[0], h[1], h[2], h[3]);
    o[1] = make_float4(l[0], l[1], l[2], l[3]);
  }
}

__global__ void split_dd_vec_kernel(long long n, const double* __restrict__ v,
                                    float* __restrict__ lo) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float h, l;
    dd_split(v[i], h, l);
    lo[i] = l;
  }
}

// (sh, sl) += (ah + al)(xh + xl).  The rounded product and sums are explicit intrinsics so that
// none is contracted into an FMA: p must be the same rounded value in the error term and the
// two-sum.
__device__ __forceinline__ void dd_fma(float& sh, float& sl, float ah, float al, float xh, float xl) {
  const float p = __fmul_rn(ah, xh);
  float e = fmaf(ah, xh, -p);   // exact: ah xh - p
  e = fmaf(ah, xl, e);
  e = fmaf(al, xh, e);
  const float s = __fadd_rn(sh, p);
  const float z = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(p, z));
  sl = __fadd_rn(sl, __fadd_rn(err, e));
  sh = s;
}

// Y = alpha (A X) + diag(delta) R (R optional), float64 in and out; b a multiple of 4, no long
// rows.  tpr = b / 4 threads per row, each four columns.
__global__ void __launch_bounds__(256) spmm_dd_kernel(
    int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
    const float* __restrict__ vh, const float* __restrict__ vl, const float* __restrict__ XD,
    int b, double* __restrict__ Y, int ldy, double alpha, const double* __restrict__ R, int ldr,
    const double* __restrict__ delta, int tpr, int rpb) {
  const int t = threadIdx.x;
  const int rl = t / tpr;
  if (rl >= rpb) return;
  const int row = blockIdx.x * rpb + rl;
  if (row >= n) return;
  const int g = t - rl * tpr, c0 = 4 * g, g4 = b >> 2;
  float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
  const int p0 = __ldg(rowptr + row), p1 = __ldg(rowptr + row + 1);
  for (int k = p0; k < p1; k += 4) {
    int j[4];
    float ah[4], al[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool ok = k + u < p1;
      j[u] = ok ? __ldg(colidx + k + u) : row;
      ah[u] = ok ? __ldg(vh + k + u) : 0.f;
      al[u] = ok ? __ldg(vl + k + u) : 0.f;
    }
    float4 xh[4], xl[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4* q = reinterpret_cast<const float4*>(XD + ((size_t)j[u] * g4 + g) * 8);
      xh[u] = __ldg(q);
      xl[u] = __ldg(q + 1);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (k + u < p1) {
        dd_fma(sh[0], sl[0], ah[u], al[u], xh[u].x, xl[u].x);
        dd_fma(sh[1], sl[1], ah[u], al[u], xh[u].y, xl[u].y);
        dd_fma(sh[2], sl[2], ah[u], al[u], xh[u].z, xl[u].z);
        dd_fma(sh[3], sl[3], ah[u], al[u], xh[u].w, xl[u].w);
      }
    }
  }
  double out[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) out[i] = alpha * ((double)sh[i] + (double)sl[i]);
  if (R != nullptr) {
#pragma unroll
    for (int i = 0; i < 4; ++i) out[i] = fma(__ldg(delta + c0 + i), R[(size_t)row * ldr + c0 + i], out[i]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) Y[(size_t)row * ldy + c0 + i] = out[i];
}

bool spmm_dd_supported(int b, const SpmmLong* lg) {
  return b >= 4 && b % 4 == 0 && b <= 128 && (lg == nullptr || lg->n_seg == 0);
}

size_t spmm_dd_scratch_floats(int n, int b) { return (size_t)n * 2 * (size_t)b + 64; }

cudaError_t launch_split_dd_vec(cudaStream_t st, long long n, const double* v, float* lo) {
  if (n <= 0) return cudaSuccess;
  const long long grid = std::min<long long>((n + 255) / 256, 16LL * kSMs);
  split_dd_vec_kernel<<<(unsigned)grid, 256, 0, st>>>(n, v, lo); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_spmm_dd(cudaStream_t st, int n, const int* rowptr, const int* colidx,
                           const float* vh, const float* vl, const double* X, int ldx, int b,
                           double* Y, int ldy, double alpha, const double* R, int ldr,
                           const double* delta, float* scratch) {
  if (n <= 0 || b <= 0) return cudaSuccess;
  if (b % 4 != 0 || b > 128) return cudaErrorInvalidValue;
  const long long items = (long long)n * (b / 4);
  const long long sg = std::min<long long>((items + 255) / 256, 16LL * kSMs);
  split_dd_kernel<<<(unsigned)sg, 256, 0, st>>>(n, b, X, ldx, scratch); note_launch();
  const int tpr = b / 4;
  const int rpb = std::max(1, 256 / tpr);
  spmm_dd_kernel<<<ceil_div(n, rpb), rpb * tpr, 0, st>>>(n, rowptr, colidx, vh, vl, scratch, b, Y,
                                                         ldy, alpha, R, ldr, delta, tpr, rpb);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_spmm_resid_dd(cudaStream_t st, int n, const int* rowptr, const int* colidx,
                                 const float* vh, const float* vl, const double* V, int ldv,
                                 int b, const double* d, double* partial, int* n_parts,
                                 double* Rout, int ldr, double* negd, float* scratch);

// ---------------- residual norms (Step 12) ----------------
// R = A V - V diag(d) through the row kernel (all rows in flight at once; the product's
// epilogue subtracts d_j v_j), then one streaming pass for the per-CTA partial sums of r_j^2
// and v_j^2 (fixed order: deterministic).
constexpr int kResidThreads = 256;

__global__ void negate_kernel(int b, const double* __restrict__ d, double* __restrict__ out) {
  for (int j = threadIdx.x; j < b; j += blockDim.x) out[j] = -d[j];
}

__global__ void __launch_bounds__(kResidThreads) resid_norms_kernel(
    int n, const double* __restrict__ R, int ldr, const double* __restrict__ V, int ldv, int b,
    double* __restrict__ partial) {
  __shared__ double s_r[kResidThreads];
  __shared__ double s_v[kResidThreads];
  const int rpb = kResidThreads / b;
  const int t = threadIdx.x;
  const int rl = t / b, c = t - rl * b;
  double r2 = 0.0, v2 = 0.0;
  if (rl < rpb)
    for (int row = blockIdx.x * rpb + rl; row < n; row += gridDim.x * rpb) {
      const double r = R[(size_t)row * ldr + c], v = V[(size_t)row * ldv + c];
      r2 = fma(r, r, r2);
      v2 = fma(v, v, v2);
    }
  s_r[t] = rl < rpb ? r2 : 0.0;
  s_v[t] = rl < rpb ? v2 : 0.0;
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
                              int ldr, double* negd, const SpmmLong* lg) {
  if (b > kResidThreads || b <= 0 || Rout == nullptr || negd == nullptr || ldr < b)
    return cudaErrorInvalidValue;
  negate_kernel<<<1, 64, 0, st>>>(b, d, negd); note_launch();
  cudaError_t e = launch_spmm_axpby<double>(st, n, rowptr, colidx, val, V, ldv, b, Rout, ldr,
                                            nullptr, 0, 1.0, 0.0, 0.0, V, ldv, negd, lg);
  if (e != cudaSuccess) return e;
  const int grid = spmm_resid_max_parts(n, b);
  *n_parts = grid;
  resid_norms_kernel<<<grid, kResidThreads, 0, st>>>(n, Rout, ldr, V, ldv, b, partial);
  note_launch();
  return cudaGetLastError();
}


cudaError_t launch_spmm_resid_dd(cudaStream_t st, int n, const int* rowptr, const int* colidx,
                                 const float* vh, const float* vl, const double* V, int ldv,
                                 int b, const double* d, double* partial, int* n_parts,
                                 double* Rout, int ldr, double* negd, float* scratch) {
  if (b > kResidThreads || b <= 0 || Rout == nullptr || negd == nullptr || ldr < b)
    return cudaErrorInvalidValue;
  negate_kernel<<<1, 64, 0, st>>>(b, d, negd); note_launch();
  cudaError_t e = launch_spmm_dd(st, n, rowptr, colidx, vh, vl, V, ldv, b, Rout, ldr, 1.0, V, ldv,
                                 negd, scratch);
  if (e != cudaSuccess) return e;
  const int grid = spmm_resid_max_parts(n, b);
  *n_parts = grid;
  resid_norms_kernel<<<grid, kResidThreads, 0, st>>>(n, Rout, ldr, V, ldv, b, partial);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bchdav
