// Algorithm 1, Steps 4 and 5 after the eigensolver: the rows of the eigenvector block scaled to
// unit length (the nodes' features) and Lloyd's k-means on them, seeded by farthest-first
// traversal.  The arithmetic is fixed so that every result is bit-reproducible and independent
// of the launch shape:
//   features   X_id = float32(V_id * r_i), r_i = 1 / sqrt(s_i), s_i = sum over d in order of
//              V_id * V_id (float64, separate multiply and add); a zero row stays zero;
//   distance   acc = 0; acc = acc + (x_d - c_d)^2 over d in order, float32, no fused multiply-add;
//   seeding    s_0 = first, s_j = argmax_i min_{l<j} dist(X_i, X_{s_l}), lowest index on ties;
//   assignment nearest float32(C_j), lowest index on ties;
//   update     C_j = float64(sum of round(X_i * 2^36) over the members, a 64-bit integer sum)
//              / count * 2^-36, the same bits in any summation order; an empty cluster keeps
//              its centroid.
// Features are stored transposed (Xt: dim x n, row-major, ld >= n) so that the per-node loops
// read each dimension with coalesced loads.  The assignment is bound by float32 arithmetic: per
// node, centroid and dimension 3 operations, issued for two centroids at a time as paired
// float32 (f32x2) instructions, the centroid pairs broadcast from shared memory.
#include <algorithm>

#include "handle.cuh"

namespace bchdav {
namespace {

constexpr int kNormRows = 32;                    // rows per normalisation tile
constexpr int kKmThreads = 256;                  // threads of the node-parallel kernels
constexpr double kQScale = 68719476736.0;        // 2^36
constexpr double kQInv = 1.0 / 68719476736.0;    // 2^-36, exact
constexpr int kMaxDim = 512;
constexpr size_t kSmemSumBytes = 48 * 1024;      // per-CTA fixed-point sums up to this size

// ---- Step 4: Xt(d, i) = float32(V(i, d) * r_i), r_i = 1 / ||V(i, :)|| (0 for a zero row)
__global__ void row_normalize_kernel(int n, int dim, const double* __restrict__ V, long long ldv,
                                     float* __restrict__ Xt, long long ldx) {
  extern __shared__ double sv[];   // kNormRows x (dim + 1)
  __shared__ double rinv[kNormRows];
  const int r0 = blockIdx.x * kNormRows;
  const int rows = min(kNormRows, n - r0);
  const int sp = dim + 1;
  for (int e = threadIdx.x; e < rows * dim; e += blockDim.x) {
    const int r = e / dim, d = e - r * dim;
    sv[r * sp + d] = V[(size_t)(r0 + r) * ldv + d];
  }
  __syncthreads();
  if (threadIdx.x < rows) {
    const double* p = sv + threadIdx.x * sp;
    double s = 0.0;
    for (int d = 0; d < dim; ++d) s = __dadd_rn(s, __dmul_rn(p[d], p[d]));
    rinv[threadIdx.x] = s > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(s)) : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kNormRows * dim; e += blockDim.x) {
    const int d = e / kNormRows, r = e - d * kNormRows;
    if (r < rows)
      Xt[(size_t)d * ldx + r0 + r] = __double2float_rn(__dmul_rn(sv[r * sp + d], rinv[r]));
  }
}

__device__ __forceinline__ float sq_step(float acc, float x, float c) {
  const float t = __fsub_rn(x, c);
  return __fadd_rn(acc, __fmul_rn(t, t));
}

// Two float32 lanes in one 64-bit register (low word first) and the lane-wise IEEE
// round-to-nearest subtract, multiply and add of sm_100-class GPUs: the same two results as
// two scalar operations, in one instruction.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t pack2(float lo, float hi) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float lo_of(f2_t v) { return __uint_as_float((unsigned)(v & 0xffffffffull)); }
__device__ __forceinline__ float hi_of(f2_t v) { return __uint_as_float((unsigned)(v >> 32)); }

// acc + (x - c)^2 in both lanes, each operation rounded to float32
__device__ __forceinline__ f2_t sq_step2(f2_t acc, f2_t x, f2_t c) {
  f2_t t, q, r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(x), "l"(c));
  asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(q) : "l"(t));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(acc), "l"(q));
  return r;
}

__device__ __forceinline__ unsigned long long max_u64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

// ---- farthest-first seeding, step j >= 1: dmin_i = min(dmin_i, dist(X_i, X_{s_{j-1}})) and
// keys[j] = max_i (bits(dmin_i) << 32 | ~i), i.e. the largest dmin, lowest index on ties
// (dmin >= 0, so its bits order like its value).
__global__ void ff_step_kernel(int n, int dim, const float* __restrict__ Xt, long long ldx,
                               float* __restrict__ dmin, unsigned long long* __restrict__ keys,
                               int j, int first) {
  extern __shared__ float cs[];   // dim
  __shared__ unsigned long long wmax[kKmThreads / 32];
  const int prev = j == 1 ? first : (int)(~(unsigned)(keys[j - 1] & 0xffffffffull));
  for (int d = threadIdx.x; d < dim; d += blockDim.x) cs[d] = Xt[(size_t)d * ldx + prev];
  __syncthreads();
  unsigned long long best = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float* xp = Xt + i;
    float acc = 0.f;
#pragma unroll 4
    for (int d = 0; d < dim; ++d) acc = sq_step(acc, xp[(size_t)d * ldx], cs[d]);
    const float m = j == 1 ? acc : fminf(dmin[i], acc);
    dmin[i] = m;
    best = max_u64(best, ((unsigned long long)__float_as_uint(m) << 32) |
                             (unsigned long long)(~(unsigned)i));
  }
  for (int o = 16; o; o >>= 1) best = max_u64(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0ull;
    for (int o = 16; o; o >>= 1) best = max_u64(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (threadIdx.x == 0) atomicMax(&keys[j], best);
  }
}

// The same step over four consecutive nodes per thread (float4 loads; needs ldx % 4 == 0 and a
// 16-byte aligned Xt; nodes n..ldx-1 of the padded rows are read and discarded).
__global__ void ff_step4_kernel(int n, int dim, const float* __restrict__ Xt, long long ldx,
                                float* __restrict__ dmin, unsigned long long* __restrict__ keys,
                                int j, int first) {
  extern __shared__ float cs[];   // dim
  __shared__ unsigned long long wmax[kKmThreads / 32];
  const int prev = j == 1 ? first : (int)(~(unsigned)(keys[j - 1] & 0xffffffffull));
  for (int d = threadIdx.x; d < dim; d += blockDim.x) cs[d] = Xt[(size_t)d * ldx + prev];
  __syncthreads();
  unsigned long long best = 0;
  const int quads = (n + 3) >> 2;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < quads; t += gridDim.x * blockDim.x) {
    const float4* xp = reinterpret_cast<const float4*>(Xt) + t;
    const long long ld4 = ldx >> 2;
    f2_t a01 = 0ull, a23 = 0ull;
#pragma unroll 8
    for (int d = 0; d < dim; ++d) {
      const float4 v = xp[(size_t)d * ld4];
      const f2_t cc = pack2(cs[d], cs[d]);
      a01 = sq_step2(a01, pack2(v.x, v.y), cc);
      a23 = sq_step2(a23, pack2(v.z, v.w), cc);
    }
    const float acc[4] = {lo_of(a01), hi_of(a01), lo_of(a23), hi_of(a23)};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = 4 * t + u;
      if (i < n) {
        const float m = j == 1 ? acc[u] : fminf(dmin[i], acc[u]);
        dmin[i] = m;
        best = max_u64(best, ((unsigned long long)__float_as_uint(m) << 32) |
                                 (unsigned long long)(~(unsigned)i));
      }
    }
  }
  for (int o = 16; o; o >>= 1) best = max_u64(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0ull;
    for (int o = 16; o; o >>= 1) best = max_u64(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (threadIdx.x == 0) atomicMax(&keys[j], best);
  }
}

__global__ void ff_seeds_kernel(int nc, int first, const unsigned long long* __restrict__ keys,
                                int* __restrict__ seeds) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nc; j += gridDim.x * blockDim.x)
    seeds[j] = j == 0 ? first : (int)(~(unsigned)(keys[j] & 0xffffffffull));
}

// ---- Lloyd's iteration
struct KmArgs {
  int n, dim, dimp, nc;
  const float* Xt;
  long long ldx;
  const float* C32;          // nc x dimp, columns dim..dimp-1 zero
  int* labels;
  unsigned long long* S;     // nc x dim fixed-point sums (two's complement)
  int* counts;               // nc
  int* changed;
  int* next_chunk;           // chunk counter of the warp-scheduled kernel (zero at launch)
  int first_round;
};

// C_j = X_{s_j}; a seed outside [0, n) sets err and reads node 0 instead.
__global__ void km_init_kernel(int n, int nc, int dim, int dimp, const float* __restrict__ Xt,
                               long long ldx, const int* __restrict__ seeds,
                               double* __restrict__ C64, float* __restrict__ C32,
                               int* __restrict__ err) {
  const long long total = (long long)nc * dimp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / dimp), d = (int)(e - (long long)c * dimp);
    int s = seeds[c];
    if (s < 0 || s >= n) {
      if (d == 0) atomicExch(err, 1);
      s = 0;
    }
    const float x = d < dim ? Xt[(size_t)d * ldx + s] : 0.f;
    C32[e] = x;
    if (d < dim) C64[(size_t)c * dim + d] = (double)x;
  }
}

// The node's fixed-point features into its cluster's sums: one shuffle-reduced atomic per
// dimension when the warp's valid nodes share a label, else one atomic per node and dimension.
__device__ __forceinline__ void km_accumulate(const float* xp, bool valid, int lab, int dim,
                                              long long ldx, unsigned long long* Sdst,
                                              int* Cdst) {
  const unsigned vm = __ballot_sync(0xffffffffu, valid);
  if (!vm) return;
  const int lane = threadIdx.x & 31;
  const int lab0 = __shfl_sync(0xffffffffu, lab, __ffs(vm) - 1);
  if (__all_sync(0xffffffffu, !valid || lab == lab0)) {
    for (int d = 0; d < dim; ++d) {
      long long q = valid ? __double2ll_rn((double)xp[(size_t)d * ldx] * kQScale) : 0ll;
      for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      if (lane == 0) atomicAdd(&Sdst[(size_t)lab0 * dim + d], (unsigned long long)q);
    }
    if (lane == 0) atomicAdd(&Cdst[lab0], __popc(vm));
  } else if (valid) {
    for (int d = 0; d < dim; ++d) {
      const long long q = __double2ll_rn((double)xp[(size_t)d * ldx] * kQScale);
      atomicAdd(&Sdst[(size_t)lab * dim + d], (unsigned long long)q);
    }
    atomicAdd(&Cdst[lab], 1);
  }
}

// Nearest centroid of each node when the centroids do not fit in shared memory at once: blocks
// of CB centroids staged in turn, CB/2 paired float32 chains per thread; label change count and
// fixed-point sums as above (in shared memory first when the sums fit).
template <int CB, bool SMEM_SUM>
__global__ void __launch_bounds__(kKmThreads) km_assign_kernel(KmArgs a) {
  static_assert(CB % 2 == 0, "centroids are processed in pairs");
  constexpr int CP = CB / 2;
  extern __shared__ __align__(16) unsigned char km_smem[];
  // centroid pairs: float (p, d, s) at (p * dimp + d) * 2 + s, centroid cb0 + 2p + s
  float* csf = reinterpret_cast<float*>(km_smem);
  const ulonglong2* cs2 = reinterpret_cast<const ulonglong2*>(km_smem);
  unsigned long long* ss =
      reinterpret_cast<unsigned long long*>(km_smem + (size_t)CB * a.dimp * sizeof(float));
  int* sc = reinterpret_cast<int*>(ss + (size_t)a.nc * a.dim);
  __shared__ int s_changed;
  const int dq4 = a.dimp >> 2;
  const int dh = a.dimp >> 1;   // 128-bit words per centroid pair
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_changed = 0;
  if (SMEM_SUM) {
    for (int e = threadIdx.x; e < a.nc * a.dim; e += kKmThreads) ss[e] = 0ull;
    for (int e = threadIdx.x; e < a.nc; e += kKmThreads) sc[e] = 0;
  }
  unsigned long long* Sdst = SMEM_SUM ? ss : a.S;
  int* Cdst = SMEM_SUM ? sc : a.counts;
  int nchg = 0;
  __syncthreads();
  for (long long base = (long long)blockIdx.x * kKmThreads; base < a.n;
       base += (long long)gridDim.x * kKmThreads) {
    const int i = (int)base + threadIdx.x;
    const bool valid = i < a.n;
    const float* xp = a.Xt + (valid ? i : a.n - 1);
    float best = __int_as_float(0x7f800000);
    int lab = 0;
    for (int cb0 = 0; cb0 < a.nc; cb0 += CB) {
      __syncthreads();
      for (int e = threadIdx.x; e < CB * a.dimp; e += kKmThreads) {
        const int c = e / a.dimp, d = e - c * a.dimp;
        csf[((c >> 1) * a.dimp + d) * 2 + (c & 1)] =
            cb0 + c < a.nc ? a.C32[(size_t)(cb0 + c) * a.dimp + d] : 0.f;
      }
      __syncthreads();
      f2_t acc[CP];
#pragma unroll
      for (int p = 0; p < CP; ++p) acc[p] = 0ull;
      for (int q = 0; q < dq4; ++q) {
        const int d = 4 * q;
        const float x0 = xp[(size_t)d * a.ldx];
        const float x1 = d + 1 < a.dim ? xp[(size_t)(d + 1) * a.ldx] : 0.f;
        const float x2 = d + 2 < a.dim ? xp[(size_t)(d + 2) * a.ldx] : 0.f;
        const float x3 = d + 3 < a.dim ? xp[(size_t)(d + 3) * a.ldx] : 0.f;
        const f2_t y0 = pack2(x0, x0), y1 = pack2(x1, x1), y2 = pack2(x2, x2), y3 = pack2(x3, x3);
#pragma unroll
        for (int p = 0; p < CP; ++p) {
          const ulonglong2 u = cs2[p * dh + 2 * q];       // dims d, d+1 of both centroids
          const ulonglong2 w = cs2[p * dh + 2 * q + 1];   // dims d+2, d+3
          f2_t t = sq_step2(acc[p], y0, u.x);
          t = sq_step2(t, y1, u.y);
          t = sq_step2(t, y2, w.x);
          acc[p] = sq_step2(t, y3, w.y);
        }
      }
#pragma unroll
      for (int p = 0; p < CP; ++p) {
        const int c = cb0 + 2 * p;
        const float a0 = lo_of(acc[p]), a1 = hi_of(acc[p]);
        if (c < a.nc && a0 < best) {
          best = a0;
          lab = c;
        }
        if (c + 1 < a.nc && a1 < best) {
          best = a1;
          lab = c + 1;
        }
      }
    }
    if (valid) {
      if (!a.first_round && a.labels[i] != lab) ++nchg;
      a.labels[i] = lab;
    }
    km_accumulate(xp, valid, lab, a.dim, a.ldx, Sdst, Cdst);
  }
  for (int o = 16; o; o >>= 1) nchg += __shfl_xor_sync(0xffffffffu, nchg, o);
  if (lane == 0 && nchg) atomicAdd(&s_changed, nchg);
  __syncthreads();
  if (threadIdx.x == 0 && s_changed) atomicAdd(a.changed, s_changed);
  if (SMEM_SUM) {
    for (int e = threadIdx.x; e < a.nc * a.dim; e += kKmThreads)
      if (ss[e]) atomicAdd(&a.S[e], ss[e]);
    for (int e = threadIdx.x; e < a.nc; e += kKmThreads)
      if (sc[e]) atomicAdd(&a.counts[e], sc[e]);
  }
}

// Assignment with every centroid resident in shared memory (padded to a multiple of CB with
// zero centroids that are never chosen).  Warps run independently: each takes 64-node chunks
// from a counter, two nodes per lane, so that one shared-memory load of a centroid pair feeds
// both nodes; the features of the next four dimensions are loaded before the current four are
// used.  Up to 20 centroids per block the registers are capped for three CTAs per SM (24 warps;
// the fastest of two and three CTAs measured at 1M nodes x 100 centroids x 100 dimensions).
template <int CB, bool SMEM_SUM>
__global__ void __launch_bounds__(kKmThreads, CB <= 20 ? 3 : 2) km_assign_all_kernel(KmArgs a) {
  static_assert(CB % 2 == 0, "centroids are processed in pairs");
  constexpr int CP = CB / 2;
  extern __shared__ __align__(16) unsigned char km_smem[];
  const int ncp = (a.nc + CB - 1) / CB * CB;
  float* csf = reinterpret_cast<float*>(km_smem);
  const ulonglong2* cs2 = reinterpret_cast<const ulonglong2*>(km_smem);
  unsigned long long* ss =
      reinterpret_cast<unsigned long long*>(km_smem + (size_t)ncp * a.dimp * sizeof(float));
  int* sc = reinterpret_cast<int*>(ss + (size_t)a.nc * a.dim);
  __shared__ int s_changed;
  const int dq4 = a.dimp >> 2;
  const int dh = a.dimp >> 1;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_changed = 0;
  for (int e = threadIdx.x; e < ncp * a.dimp; e += kKmThreads) {
    const int c = e / a.dimp, d = e - c * a.dimp;
    csf[((c >> 1) * a.dimp + d) * 2 + (c & 1)] = c < a.nc ? a.C32[(size_t)c * a.dimp + d] : 0.f;
  }
  if (SMEM_SUM) {
    for (int e = threadIdx.x; e < a.nc * a.dim; e += kKmThreads) ss[e] = 0ull;
    for (int e = threadIdx.x; e < a.nc; e += kKmThreads) sc[e] = 0;
  }
  unsigned long long* Sdst = SMEM_SUM ? ss : a.S;
  int* Cdst = SMEM_SUM ? sc : a.counts;
  int nchg = 0;
  __syncthreads();
  for (;;) {
    int chunk = 0;
    if (lane == 0) chunk = atomicAdd(a.next_chunk, 1);
    chunk = __shfl_sync(0xffffffffu, chunk, 0);
    const long long base = (long long)chunk * 64;
    if (base >= a.n) break;
    const int i0 = (int)base + lane, i1 = i0 + 32;
    const bool v0 = i0 < a.n, v1 = i1 < a.n;
    const float* xa = a.Xt + (v0 ? i0 : a.n - 1);
    const float* xb = a.Xt + (v1 ? i1 : a.n - 1);
    float best0 = __int_as_float(0x7f800000), best1 = best0;
    int lab0 = 0, lab1 = 0;
    for (int cb0 = 0; cb0 < ncp; cb0 += CB) {
      const ulonglong2* cp = cs2 + (size_t)(cb0 >> 1) * dh;
      f2_t acc0[CP], acc1[CP];
#pragma unroll
      for (int p = 0; p < CP; ++p) acc0[p] = acc1[p] = 0ull;
      float na[4], nb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        na[u] = u < a.dim ? xa[(size_t)u * a.ldx] : 0.f;
        nb[u] = u < a.dim ? xb[(size_t)u * a.ldx] : 0.f;
      }
      for (int q = 0; q < dq4; ++q) {
        const f2_t y0 = pack2(na[0], na[0]), y1 = pack2(na[1], na[1]);
        const f2_t y2 = pack2(na[2], na[2]), y3 = pack2(na[3], na[3]);
        const f2_t z0 = pack2(nb[0], nb[0]), z1 = pack2(nb[1], nb[1]);
        const f2_t z2 = pack2(nb[2], nb[2]), z3 = pack2(nb[3], nb[3]);
        const int dn = 4 * q + 4;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          na[u] = dn + u < a.dim ? xa[(size_t)(dn + u) * a.ldx] : 0.f;
          nb[u] = dn + u < a.dim ? xb[(size_t)(dn + u) * a.ldx] : 0.f;
        }
#pragma unroll
        for (int p = 0; p < CP; ++p) {
          const ulonglong2 u = cp[p * dh + 2 * q];       // dims 4q, 4q+1 of both centroids
          const ulonglong2 w = cp[p * dh + 2 * q + 1];   // dims 4q+2, 4q+3
          f2_t t = sq_step2(acc0[p], y0, u.x);
          t = sq_step2(t, y1, u.y);
          t = sq_step2(t, y2, w.x);
          acc0[p] = sq_step2(t, y3, w.y);
          t = sq_step2(acc1[p], z0, u.x);
          t = sq_step2(t, z1, u.y);
          t = sq_step2(t, z2, w.x);
          acc1[p] = sq_step2(t, z3, w.y);
        }
      }
#pragma unroll
      for (int p = 0; p < CP; ++p) {
        const int c = cb0 + 2 * p;
        if (c < a.nc) {
          if (lo_of(acc0[p]) < best0) { best0 = lo_of(acc0[p]); lab0 = c; }
          if (lo_of(acc1[p]) < best1) { best1 = lo_of(acc1[p]); lab1 = c; }
        }
        if (c + 1 < a.nc) {
          if (hi_of(acc0[p]) < best0) { best0 = hi_of(acc0[p]); lab0 = c + 1; }
          if (hi_of(acc1[p]) < best1) { best1 = hi_of(acc1[p]); lab1 = c + 1; }
        }
      }
    }
    if (v0) {
      if (!a.first_round && a.labels[i0] != lab0) ++nchg;
      a.labels[i0] = lab0;
    }
    if (v1) {
      if (!a.first_round && a.labels[i1] != lab1) ++nchg;
      a.labels[i1] = lab1;
    }
    km_accumulate(xa, v0, lab0, a.dim, a.ldx, Sdst, Cdst);
    km_accumulate(xb, v1, lab1, a.dim, a.ldx, Sdst, Cdst);
  }
  for (int o = 16; o; o >>= 1) nchg += __shfl_xor_sync(0xffffffffu, nchg, o);
  if (lane == 0 && nchg) atomicAdd(&s_changed, nchg);
  __syncthreads();
  if (threadIdx.x == 0 && s_changed) atomicAdd(a.changed, s_changed);
  if (SMEM_SUM) {
    for (int e = threadIdx.x; e < a.nc * a.dim; e += kKmThreads)
      if (ss[e]) atomicAdd(&a.S[e], ss[e]);
    for (int e = threadIdx.x; e < a.nc; e += kKmThreads)
      if (sc[e]) atomicAdd(&a.counts[e], sc[e]);
  }
}

// C_j = float64(Q_j) / count_j * 2^-36 where count_j > 0; the sums are cleared for the next round.
__global__ void km_update_kernel(int nc, int dim, int dimp, unsigned long long* __restrict__ S,
                                 const int* __restrict__ counts, double* __restrict__ C64,
                                 float* __restrict__ C32) {
  const long long total = (long long)nc * dim;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / dim), d = (int)(e - (long long)c * dim);
    const int cnt = counts[c];
    if (cnt > 0) {
      const double m =
          __dmul_rn(__ddiv_rn(__ll2double_rn((long long)S[e]), (double)cnt), kQInv);
      C64[e] = m;
      C32[(size_t)c * dimp + d] = __double2float_rn(m);
    }
    S[e] = 0ull;
  }
}

// Centroid block: the candidate that pads nc least, the larger one on ties.
int pick_cb(int nc) {
  static const int cand[] = {32, 28, 24, 20, 16, 12, 8, 4};
  int best = 32, pad = 1 << 30;
  for (int cb : cand) {
    const int p = (nc + cb - 1) / cb * cb;
    if (p < pad) {
      pad = p;
      best = cb;
    }
  }
  return best;
}

constexpr size_t kAllCentroidsBytes = 96 * 1024;   // centroids resident in shared memory

template <typename K>
cudaError_t launch_persistent(K k, const KmArgs& a, size_t smem, long long max_ctas, int sms,
                              cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kKmThreads, smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::max<long long>(
      1, std::min<long long>(max_ctas, (long long)sms * std::max(per_sm, 1)));
  k<<<grid, kKmThreads, smem, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

template <int CB>
cudaError_t launch_assign_cb(const KmArgs& a, int sms, cudaStream_t st) {
  const size_t sums = (size_t)a.nc * a.dim * 8 + (size_t)a.nc * 4;
  const bool smem_sum = sums <= kSmemSumBytes;
  const size_t all = (size_t)((a.nc + CB - 1) / CB * CB) * a.dimp * sizeof(float);
  if (all + (smem_sum ? sums : 0) <= kAllCentroidsBytes) {
    const long long chunks = ((long long)a.n + 63) / 64;
    // the chunk counter belongs to this launch alone: cleared before it on the stream
    cudaError_t e = cudaMemsetAsync(a.next_chunk, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (smem_sum)
      return launch_persistent(km_assign_all_kernel<CB, true>, a, all + sums, chunks, sms, st);
    return launch_persistent(km_assign_all_kernel<CB, false>, a, all, chunks, sms, st);
  }
  const size_t base = (size_t)CB * a.dimp * sizeof(float);
  const long long tiles = ((long long)a.n + kKmThreads - 1) / kKmThreads;
  if (smem_sum)
    return launch_persistent(km_assign_kernel<CB, true>, a, base + sums, tiles, sms, st);
  return launch_persistent(km_assign_kernel<CB, false>, a, base, tiles, sms, st);
}

cudaError_t launch_assign(const KmArgs& a, int sms, cudaStream_t st) {
  switch (pick_cb(a.nc)) {
    case 4: return launch_assign_cb<4>(a, sms, st);
    case 8: return launch_assign_cb<8>(a, sms, st);
    case 12: return launch_assign_cb<12>(a, sms, st);
    case 16: return launch_assign_cb<16>(a, sms, st);
    case 20: return launch_assign_cb<20>(a, sms, st);
    case 24: return launch_assign_cb<24>(a, sms, st);
    case 28: return launch_assign_cb<28>(a, sms, st);
    default: return launch_assign_cb<32>(a, sms, st);
  }
}

int grid_for(long long items, int sms) {
  return (int)std::max<long long>(1, std::min<long long>((items + kKmThreads - 1) / kKmThreads,
                                                         (long long)sms * 8));
}

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// Workspace of one clustering call, carved from h->km.
struct KmWork {
  float* C32;
  double* C64;
  unsigned long long* S;
  int* counts;
  int* flags;   // [0] labels changed this round, [1] chunk counter, [2] invalid seed
  unsigned long long* keys;
  int* seeds;
  float* dmin;
};

size_t km_bytes(int n, int dim, int nc) {
  const int dimp = round_up(dim, 4);
  return al256((size_t)nc * dimp * 4) + al256((size_t)nc * dim * 8) * 2 + al256((size_t)nc * 4) +
         al256(16) + al256((size_t)nc * 8) + al256((size_t)nc * 4) + al256((size_t)n * 4);
}

KmWork km_carve(void* p, int n, int dim, int nc) {
  const int dimp = round_up(dim, 4);
  char* c = static_cast<char*>(p);
  KmWork w;
  w.C32 = reinterpret_cast<float*>(c);
  c += al256((size_t)nc * dimp * 4);
  w.C64 = reinterpret_cast<double*>(c);
  c += al256((size_t)nc * dim * 8);
  w.S = reinterpret_cast<unsigned long long*>(c);
  c += al256((size_t)nc * dim * 8);
  w.counts = reinterpret_cast<int*>(c);
  c += al256((size_t)nc * 4);
  w.flags = reinterpret_cast<int*>(c);
  c += al256(16);
  w.keys = reinterpret_cast<unsigned long long*>(c);
  c += al256((size_t)nc * 8);
  w.seeds = reinterpret_cast<int*>(c);
  c += al256((size_t)nc * 4);
  w.dmin = reinterpret_cast<float*>(c);
  return w;
}

#define HCUDA(expr) BCHDAV_CUDA_OK(expr, h)

bchdav_status check_features(bchdav_handle h, int32_t n, int32_t dim, int32_t nc,
                             int64_t ldx) {
  if (n < 1 || n >= (1 << 27) || dim < 1 || dim > kMaxDim || nc < 1 || nc > n || ldx < n) {
    h->set_error(BCHDAV_ERR_ARG, "clustering: need 1 <= n < 2^27, 1 <= dim <= 512, "
                                 "1 <= n_clusters <= n and ldx >= n");
    return BCHDAV_ERR_ARG;
  }
  return BCHDAV_OK;
}

// Farthest-first seeds.  padded: the rows of Xt may be read up to round_up(n, 4) (the float4
// path then also needs ldx % 4 == 0 and a 16-byte aligned Xt).
bchdav_status seed(bchdav_handle h, int n, int dim, const float* Xt, long long ldx, int nc,
                   int first, const KmWork& w, int* seeds, bool padded) {
  cudaStream_t st = h->stream;
  HCUDA(cudaMemsetAsync(w.keys, 0, (size_t)nc * 8, st));
  const size_t smem = (size_t)dim * sizeof(float);
  const bool vec = padded && ldx % 4 == 0 && (reinterpret_cast<uintptr_t>(Xt) & 15) == 0;
  const int grid = grid_for(vec ? (n + 3) / 4 : n, h->sms);
  for (int j = 1; j < nc; ++j) {
    if (vec)
      ff_step4_kernel<<<grid, kKmThreads, smem, st>>>(n, dim, Xt, ldx, w.dmin, w.keys, j, first);
    else
      ff_step_kernel<<<grid, kKmThreads, smem, st>>>(n, dim, Xt, ldx, w.dmin, w.keys, j, first);
    note_launch();
  }
  ff_seeds_kernel<<<(nc + 255) / 256, 256, 0, st>>>(nc, first, w.keys, seeds);
  note_launch();
  HCUDA(cudaGetLastError());
  return BCHDAV_OK;
}

bchdav_status lloyd(bchdav_handle h, int n, int dim, const float* Xt, long long ldx, int nc,
                    const int* seeds, int max_rounds, int* labels, double* centroids,
                    int32_t* rounds_out, const KmWork& w) {
  cudaStream_t st = h->stream;
  const int dimp = round_up(dim, 4);
  BCHDAV_TRY(h->ensure_aux(2));
  int* flags_host = reinterpret_cast<int*>(h->host_aux);
  HCUDA(cudaMemsetAsync(w.C32, 0, (size_t)nc * dimp * 4, st));
  HCUDA(cudaMemsetAsync(w.S, 0, (size_t)nc * dim * 8, st));
  HCUDA(cudaMemsetAsync(w.counts, 0, (size_t)nc * 4, st));
  HCUDA(cudaMemsetAsync(w.flags, 0, 16, st));
  km_init_kernel<<<grid_for((long long)nc * dimp, h->sms), kKmThreads, 0, st>>>(
      n, nc, dim, dimp, Xt, ldx, seeds, w.C64, w.C32, w.flags + 2);
  note_launch();
  HCUDA(cudaGetLastError());
  KmArgs a{n, dim, dimp, nc, Xt, ldx, w.C32, labels, w.S, w.counts, w.flags, w.flags + 1, 1};
  HCUDA(launch_assign(a, h->sms, st));
  int rounds = 1;
  a.first_round = 0;
  bool bad_seed = false;
  while (rounds < max_rounds) {
    km_update_kernel<<<grid_for((long long)nc * dim, h->sms), kKmThreads, 0, st>>>(
        nc, dim, dimp, w.S, w.counts, w.C64, w.C32);
    note_launch();
    HCUDA(cudaGetLastError());
    HCUDA(cudaMemsetAsync(w.counts, 0, (size_t)nc * 4, st));
    HCUDA(cudaMemsetAsync(w.flags, 0, 4, st));
    HCUDA(launch_assign(a, h->sms, st));
    ++rounds;
    HCUDA(cudaMemcpyAsync(flags_host, w.flags, 12, cudaMemcpyDeviceToHost, st));
    HCUDA(cudaStreamSynchronize(st));
    if (flags_host[2]) {
      bad_seed = true;
      break;
    }
    if (flags_host[0] == 0) break;
  }
  if (centroids)
    HCUDA(cudaMemcpyAsync(centroids, w.C64, (size_t)nc * dim * 8, cudaMemcpyDeviceToDevice, st));
  HCUDA(cudaMemcpyAsync(flags_host, w.flags, 12, cudaMemcpyDeviceToHost, st));
  HCUDA(cudaStreamSynchronize(st));
  if (bad_seed || flags_host[2]) {
    h->set_error(BCHDAV_ERR_ARG, "k-means: a seed index is outside [0, n)");
    return BCHDAV_ERR_ARG;
  }
  if (rounds_out) *rounds_out = rounds;
  return BCHDAV_OK;
}

}  // namespace
}  // namespace bchdav

using namespace bchdav;

extern "C" {

bchdav_status bchdav_row_normalize(bchdav_handle h, int32_t n, int32_t dim, const double* V,
                                   int64_t ldv, float* Xt, int64_t ldx) {
  if (!h) return BCHDAV_ERR_ARG;
  if (n < 1 || dim < 1 || dim > kMaxDim || ldv < dim || ldx < n || !V || !Xt) {
    h->set_error(BCHDAV_ERR_ARG, "row_normalize: need n >= 1, 1 <= dim <= 512, ldv >= dim, "
                                 "ldx >= n");
    return BCHDAV_ERR_ARG;
  }
  const size_t smem = (size_t)kNormRows * (dim + 1) * sizeof(double);
  HCUDA(cudaFuncSetAttribute(row_normalize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem));
  row_normalize_kernel<<<(n + kNormRows - 1) / kNormRows, kKmThreads, smem, h->stream>>>(
      n, dim, V, ldv, Xt, ldx);
  note_launch();
  HCUDA(cudaGetLastError());
  return BCHDAV_OK;
}

bchdav_status bchdav_kmeans_seed(bchdav_handle h, int32_t n, int32_t dim, const float* Xt,
                                 int64_t ldx, int32_t n_clusters, int32_t first, int32_t* seeds) {
  if (!h) return BCHDAV_ERR_ARG;
  BCHDAV_TRY(check_features(h, n, dim, n_clusters, ldx));
  if (!Xt || !seeds || first < 0 || first >= n) {
    h->set_error(BCHDAV_ERR_ARG, "kmeans_seed: first must lie in [0, n)");
    return BCHDAV_ERR_ARG;
  }
  BCHDAV_TRY(h->ensure(h->km, km_bytes(n, dim, n_clusters)));
  const KmWork w = km_carve(h->km.p, n, dim, n_clusters);
  return seed(h, n, dim, Xt, ldx, n_clusters, first, w, seeds, n % 4 == 0);
}

bchdav_status bchdav_kmeans(bchdav_handle h, int32_t n, int32_t dim, const float* Xt, int64_t ldx,
                            int32_t n_clusters, const int32_t* seeds, int32_t max_rounds,
                            int32_t* labels, double* centroids, int32_t* rounds) {
  if (!h) return BCHDAV_ERR_ARG;
  BCHDAV_TRY(check_features(h, n, dim, n_clusters, ldx));
  if (!Xt || !seeds || !labels || max_rounds < 1) {
    h->set_error(BCHDAV_ERR_ARG, "kmeans: need features, seeds, labels and max_rounds >= 1");
    return BCHDAV_ERR_ARG;
  }
  BCHDAV_TRY(h->ensure(h->km, km_bytes(n, dim, n_clusters)));
  const KmWork w = km_carve(h->km.p, n, dim, n_clusters);
  return lloyd(h, n, dim, Xt, ldx, n_clusters, seeds, max_rounds, labels, centroids, rounds, w);
}

bchdav_status bchdav_spectral_cluster(bchdav_handle h, int32_t n, int32_t dim, const double* V,
                                      int64_t ldv, int32_t n_clusters, int32_t first,
                                      int32_t max_rounds, int32_t* labels, double* centroids,
                                      int32_t* seeds, int32_t* rounds) {
  if (!h) return BCHDAV_ERR_ARG;
  BCHDAV_TRY(check_features(h, n, dim, n_clusters, n));
  if (!V || !labels || ldv < dim || max_rounds < 1 || first < 0 || first >= n) {
    h->set_error(BCHDAV_ERR_ARG, "spectral_cluster: need V, labels, ldv >= dim, "
                                 "max_rounds >= 1 and first in [0, n)");
    return BCHDAV_ERR_ARG;
  }
  const long long ldx = round_up(n, 4);   // rows padded for the float4 seeding pass
  BCHDAV_TRY(h->ensure(h->km_x, (size_t)ldx * dim * sizeof(float)));
  BCHDAV_TRY(h->ensure(h->km, km_bytes(n, dim, n_clusters)));
  const KmWork w = km_carve(h->km.p, n, dim, n_clusters);
  float* Xt = h->km_x.as<float>();
  BCHDAV_TRY(bchdav_row_normalize(h, n, dim, V, ldv, Xt, ldx));
  int* sd = seeds ? seeds : w.seeds;
  BCHDAV_TRY(seed(h, n, dim, Xt, ldx, n_clusters, first, w, sd, true));
  return lloyd(h, n, dim, Xt, ldx, n_clusters, sd, max_rounds, labels, centroids, rounds, w);
}

}  // extern "C"
