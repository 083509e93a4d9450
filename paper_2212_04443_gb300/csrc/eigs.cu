// Step 9 of Algorithm 2 for small H (n <= kEsMaxN): the eigendecomposition is computed in
// float32 and refined in float64.
//
// GB300's float64 pipe issues about 1.7 fused multiply-adds per clock per SM, with ~64 cycles
// between dependent operations; float32 is ~70 times faster on both counts.  A float64
// eigensolver for n of a few tens spends its time in chains of dependent float64 operations
// (0.25-2.7 ms per call at n = 8-64), so here:
//
//  1. Every CTA of one 16-CTA cluster computes, redundantly and bit-identically, an approximate
//     decomposition H ~ X diag(lam) X^T in float32 (H scaled by a power of two near ||H||_F):
//     Householder tridiagonalisation T = Q^T H Q, multisection on Sturm counts of T,
//     inverse iteration (T - lam I = L D L^T with a pivot floor, two solves from a fixed
//     pseudo-random start), classical Gram-Schmidt applied twice inside each group of
//     eigenvalues closer than 1e-3 ||T||, and X = Q Z.
//  2. The cluster refines X in float64 by the iteration of Ogita and Aishima (Japan J. Indust.
//     Appl. Math. 35, 2018), each CTA owning every 16th column and pushing what it computes to
//     the other CTAs' shared memory:
//        R = I - X^T X,  S = X^T H X,  lam_j = s_jj / (1 - r_jj),
//        delta = 2 (||S - diag(lam)||_F + ||H||_F ||R||_F),
//        E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i)   where |lam_j - lam_i| > delta,
//        E_ij = r_ij / 2                                 otherwise (and on the diagonal),
//        X <- X + X E.
//     For a pair i < j only E_ij comes from the formula and E_ji = r_ij - E_ij, so that
//     E + E^T = R holds to rounding: X stays orthonormal to float64 accuracy even where a
//     small gap makes E_ij itself ill-conditioned.  The iteration converges quadratically and
//     stops once max |E| <= 1e-8 (at most kEsMaxIt updates); the eigenvalues are the last
//     Rayleigh quotients lam_j, correct to O(max |E|^2) ||H||.
//
// The result is kept when the last update was at most 1e-7 and every pair still inside a
// cluster is uncoupled to the level a backward-stable eigensolver leaves (|s_ij| <= 4e-15 n
// ||H||_F: a degenerate eigenvalue, whose vectors may be any orthonormal basis of its space);
// otherwise (a cluster of distinct eigenvalues closer than float32 resolves, which the
// iteration leaves mixed), or for a non-finite H, a device word asks the Jacobi kernel that
// follows to replace it.
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace bchdav {
namespace {

constexpr int kEsCl = 16;          // CTAs per cluster (non-portable size, checked at set-up)
constexpr int kEsThreads = 512;
constexpr int kEsWarps = kEsThreads / 32;
constexpr int kEsMaxOwn = (kEsMaxN + kEsCl - 1) / kEsCl;
constexpr int kEsMaxIt = 6;
constexpr double kEsStop = 1e-8;
constexpr double kEsAccept = 1e-7;
constexpr double kEsCouple = 4e-15;   // x n: the coupling a backward-stable result may keep

// control words (the first doubles of the route's work area)
struct EsCtl {
  int run_jacobi;   // nonzero: the result is to be replaced by the Jacobi kernel
  int iters;        // refinement updates applied
};

__host__ __device__ inline int es_ld(int n) { return n | 1; }   // odd strides: no bank conflicts

struct EsSmem {
  double *H, *X, *Xn, *E;          // n x ld each (row-major; column j of X is vector j)
  double *P, *S, *G;               // n x kEsMaxOwn: own columns of H X, X^T H X, X^T X
  double *lam, *sS, *sR, *sE, *sC;  // lam[n]; per-CTA partials [kEsCl]
  double *own, *red;               // own lam / partial sums [3 kEsMaxOwn]; reductions [40]
  float *A, *L;                    // float32 phase: A (n x ldf) inside Xn, L (2 n x n) inside E
  float *V, *Z;                    // reflectors (row j = v_j), eigenvectors: n x ldf each
  float *tau, *d, *e, *e2, *lo, *hi, *lp, *p, *misc;
  int *cnt, *grp;
};

__host__ __device__ inline size_t es_smem_bytes(int n) {
  const size_t ld = es_ld(n), nn = (size_t)n * ld;
  const size_t dbl = 4 * nn + 3 * (size_t)n * kEsMaxOwn + n + 4 * kEsCl + 3 * kEsMaxOwn + 40;
  const size_t flt = 2 * nn + 9 * (size_t)n + 8;
  const size_t ints = 2 * (size_t)kEsThreads + n;
  return dbl * sizeof(double) + flt * sizeof(float) + ints * sizeof(int) + 16;
}

__device__ inline EsSmem es_smem(void* base, int n) {
  const size_t ld = es_ld(n), nn = (size_t)n * ld;
  EsSmem s;
  double* q = static_cast<double*>(base);
  s.H = q;
  s.X = s.H + nn;
  s.Xn = s.X + nn;
  s.E = s.Xn + nn;
  s.P = s.E + nn;
  s.S = s.P + (size_t)n * kEsMaxOwn;
  s.G = s.S + (size_t)n * kEsMaxOwn;
  s.lam = s.G + (size_t)n * kEsMaxOwn;
  s.sS = s.lam + n;
  s.sR = s.sS + kEsCl;
  s.sE = s.sR + kEsCl;
  s.sC = s.sE + kEsCl;
  s.own = s.sC + kEsCl;
  s.red = s.own + 3 * kEsMaxOwn;
  float* f = reinterpret_cast<float*>(s.red + 40);
  s.A = reinterpret_cast<float*>(s.Xn);   // n x ld floats fit in n x ld doubles
  s.L = reinterpret_cast<float*>(s.E);    // 2 n x n floats fit in n x ld doubles
  s.V = f;
  s.Z = s.V + nn;
  s.tau = s.Z + nn;
  s.d = s.tau + n;
  s.e = s.d + n;
  s.e2 = s.e + n;
  s.lo = s.e2 + n;
  s.hi = s.lo + n;
  s.lp = s.hi + n;
  s.p = s.lp + n;
  s.misc = s.p + n;                         // gl, gu, tn, pivmin
  s.cnt = reinterpret_cast<int*>(s.misc + 8 + n);
  s.grp = s.cnt + 2 * kEsThreads;
  return s;
}

__device__ __forceinline__ float wsum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float wmin_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float wmax_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double wsum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// maximum that keeps a NaN (fmax would drop it)
__device__ __forceinline__ double nanmax(double a, double b) { return (b != b || b > a) ? b : a; }
__device__ __forceinline__ double wmax_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum in a fixed order; every thread gets the result.  The float64 pipe issues
// ~1.7 operations per clock per SM, so the last stage runs in one warp, not in every thread.
__device__ double es_block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = wsum_d(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < kEsWarps ? red[lane] : 0.0;
#pragma unroll
    for (int o = kEsWarps / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[kEsWarps] = s;
  }
  __syncthreads();
  return red[kEsWarps];
}

// ---------------------------------------------------------------------------------------------
// Float32 phase (every CTA, identical): the reflectors of H's tridiagonalisation (sm.V,
// sm.tau) and the eigenvectors of T (sm.Z, n x ldf)
// ---------------------------------------------------------------------------------------------
__device__ void es_float32_phase(const EsSmem& sm, int n, double scale) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int ld = es_ld(n), ldf = ld;
  float* A = sm.A;
  for (int idx = t; idx < n * n; idx += kEsThreads) {
    const int i = idx / n, j = idx - i * n;
    A[i * ldf + j] = (float)(sm.H[i * ld + j] * scale);
  }
  __syncthreads();

  // Householder: P_j = I - tau_j v_j v_j^T on rows/columns j+1 .. n-1; A <- P_j A P_j as
  // A' -= v w^T + w v^T, p = tau A' v, w = p - (tau/2)(v^T p) v
  for (int j = 0; j + 2 < n; ++j) {
    const int r = n - j - 1;
    if (warp == 0) {
      const float x0 = A[(j + 1) * ldf + j];
      const float xa = (lane >= 1 && lane < r) ? A[(j + 1 + lane) * ldf + j] : 0.f;
      const float xb = (lane + 32 < r) ? A[(j + 1 + lane + 32) * ldf + j] : 0.f;
      const float st = wsum_f(fmaf(xa, xa, xb * xb));
      float tau = 0.f, alpha = x0, v0 = 0.f;
      if (st > 0.f) {
        alpha = -copysignf(sqrtf(fmaf(x0, x0, st)), x0);
        v0 = x0 - alpha;
        tau = 1.f / (alpha * (alpha - x0));
      }
      if (lane < r) sm.V[j * ldf + lane] = lane == 0 ? v0 : xa;
      if (lane + 32 < r) sm.V[j * ldf + lane + 32] = xb;
      if (lane == 0) {
        sm.tau[j] = tau;
        sm.e[j] = alpha;
        sm.d[j] = A[j * ldf + j];
      }
    }
    __syncthreads();
    const float tau = sm.tau[j];
    if (tau == 0.f) continue;   // uniform: the column is already reduced
    const float* v = sm.V + j * ldf;
    float* B = A + (j + 1) * ldf + (j + 1);
    const int a = t >> 3, b0 = t & 7;   // eight threads per row of the trailing block
    {
      float s = 0.f;
      if (a < r)
        for (int k = b0; k < r; k += 8) s = fmaf(B[a * ldf + k], v[k], s);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      if (a < r && b0 == 0) sm.p[a] = tau * s;
    }
    __syncthreads();
    float kp = lane < r ? v[lane] * sm.p[lane] : 0.f;
    if (lane + 32 < r) kp = fmaf(v[lane + 32], sm.p[lane + 32], kp);
    const float K = 0.5f * tau * wsum_f(kp);
    if (a < r) {
      const float va = v[a], wa = fmaf(-K, va, sm.p[a]);
      for (int b = b0; b < r; b += 8) {
        const float wb = fmaf(-K, v[b], sm.p[b]);
        B[a * ldf + b] -= fmaf(va, wb, wa * v[b]);
      }
    }
    __syncthreads();
  }
  if (t == 0) {
    sm.d[n - 2] = A[(n - 2) * ldf + (n - 2)];
    sm.d[n - 1] = A[(n - 1) * ldf + (n - 1)];
    sm.e[n - 2] = A[(n - 1) * ldf + (n - 2)];
  }
  __syncthreads();

  // Gershgorin interval, pivot floor
  float* misc = sm.misc;
  if (warp == 0) {
    float lo = FLT_MAX, hi = -FLT_MAX, em = 0.f;
    for (int i = lane; i < n; i += 32) {
      const float el = i > 0 ? fabsf(sm.e[i - 1]) : 0.f, er = i + 1 < n ? fabsf(sm.e[i]) : 0.f;
      lo = fminf(lo, sm.d[i] - (el + er));
      hi = fmaxf(hi, sm.d[i] + (el + er));
      if (i + 1 < n) em = fmaxf(em, er * er);
    }
    lo = wmin_f(lo);
    hi = wmax_f(hi);
    em = wmax_f(em);
    const float tn = fmaxf(fmaxf(fabsf(lo), fabsf(hi)), FLT_MIN);
    const float pad = 4.f * FLT_EPSILON * tn * (float)n;
    if (lane == 0) {
      misc[0] = lo - pad;
      misc[1] = hi + pad;
      misc[2] = tn;
      misc[3] = FLT_MIN * fmaxf(1.f, em);
    }
  }
  for (int i = t; i + 1 < n; i += kEsThreads) sm.e2[i] = sm.e[i] * sm.e[i];
  __syncthreads();
  const float gl = misc[0], gu = misc[1], tn = misc[2], pivmin = misc[3];
  for (int k = t; k < n; k += kEsThreads) {
    sm.lo[k] = gl;
    sm.hi[k] = gu;
  }
  __syncthreads();

  // multisection: P points per eigenvalue and round, four per thread; the points below
  // eigenvalue k (Sturm count <= k) are counted with shared-memory atomics: with counts
  // non-decreasing in x that number is the index of the first point above it
  const int tpe = kEsThreads / n;             // threads per eigenvalue (>= 8 for n <= 64)
  const int P = 4 * tpe;
  const int rounds = (int)ceilf(16.7f / logf((float)(P + 1)));   // width / (P+1)^rounds < 2^-24
  int* below = sm.cnt;
  if (t < n) below[t] = 0;
  __syncthreads();
  for (int rd = 0; rd < rounds; ++rd) {
    const int k = t / tpe, p0 = 4 * (t - k * tpe);
    if (k < n) {
      const float lo = sm.lo[k], w = (sm.hi[k] - lo) / (float)(P + 1);
      float x[4], q[4];
      int c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x[u] = fmaf(w, (float)(p0 + 1 + u), lo);
        q[u] = sm.d[0] - x[u];
        if (fabsf(q[u]) < pivmin) q[u] = -pivmin;
        c[u] = q[u] < 0.f;
      }
      for (int i = 1; i < n; ++i) {
        const float di = sm.d[i], ei = sm.e2[i - 1];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          q[u] = (di - x[u]) - __fdividef(ei, q[u]);
          if (fabsf(q[u]) < pivmin) q[u] = -pivmin;
          c[u] += q[u] < 0.f;
        }
      }
      const int nb = (c[0] <= k) + (c[1] <= k) + (c[2] <= k) + (c[3] <= k);
      if (nb) atomicAdd(&below[k], nb);
    }
    __syncthreads();
    if (t < n) {
      const float lo = sm.lo[t], w = (sm.hi[t] - lo) / (float)(P + 1);
      const int p = below[t];
      below[t] = 0;
      if (p < P) sm.hi[t] = fmaf(w, (float)(p + 1), lo);
      if (p > 0) sm.lo[t] = fmaf(w, (float)p, lo);
    }
    __syncthreads();
  }

  // shifts (equal ones separated), groups of close eigenvalues
  if (t == 0) {
    const float sep = 16.f * FLT_EPSILON * tn, gtol = 1e-3f * tn;
    float prev = 0.5f * (sm.lo[0] + sm.hi[0]);
    sm.lp[0] = prev;
    sm.grp[0] = 0;
    for (int k = 1; k < n; ++k) {
      const float lk = 0.5f * (sm.lo[k] + sm.hi[k]);
      const float lprev = 0.5f * (sm.lo[k - 1] + sm.hi[k - 1]);
      sm.grp[k] = (lk - lprev <= gtol) ? sm.grp[k - 1] : k;
      prev = fmaxf(lk, prev + sep);
      sm.lp[k] = prev;
    }
  }
  __syncthreads();

  // inverse iteration, one thread per eigenvalue: T - s I = L D L^T (unit lower bidiagonal L
  // with L_{i,i-1} = l_i, D = diag(q), |q_i| >= FLT_EPSILON ||T||), two solves
  float* Z = sm.Z;
  if (t < n) {
    const int k = t;
    const float s = sm.lp[k], floor_q = FLT_EPSILON * tn;
    float* rq = sm.L;               // 1 / q_i at [i n + k]
    float* ll = sm.L + n * n;       // l_i at [i n + k]
    float q = sm.d[0] - s;
    if (fabsf(q) < floor_q) q = copysignf(floor_q, q);
    float rp = __frcp_rn(q);
    rq[k] = rp;
    for (int i = 1; i < n; ++i) {
      const float l = sm.e[i - 1] * rp;
      q = fmaf(-l, sm.e[i - 1], sm.d[i] - s);
      if (fabsf(q) < floor_q) q = copysignf(floor_q, q);
      rp = __frcp_rn(q);
      ll[i * n + k] = l;
      rq[i * n + k] = rp;
    }
    for (int i = 0; i < n; ++i) {
      const unsigned hsh = (unsigned)(i * 7919 + k * 104729 + 17) % 2003u;
      Z[i * ldf + k] = (float)hsh * (1.f / 1001.5f) - 1.f;
    }
    for (int it = 0; it < 2; ++it) {
      float y = Z[k];
#pragma unroll 8
      for (int i = 1; i < n; ++i) {
        y = fmaf(-ll[i * n + k], y, Z[i * ldf + k]);
        Z[i * ldf + k] = y;
      }
      float z = Z[(n - 1) * ldf + k] * rq[(n - 1) * n + k];
      Z[(n - 1) * ldf + k] = z;
      float zm = fabsf(z);
#pragma unroll 8
      for (int i = n - 2; i >= 0; --i) {
        z = fmaf(-ll[(i + 1) * n + k], z, Z[i * ldf + k] * rq[i * n + k]);
        Z[i * ldf + k] = z;
        zm = fmaxf(zm, fabsf(z));
      }
      const float sc = zm > 0.f ? 1.f / zm : 1.f;
#pragma unroll 8
      for (int i = 0; i < n; ++i) Z[i * ldf + k] *= sc;
    }
    float nrm = 0.f;
    for (int i = 0; i < n; ++i) nrm = fmaf(Z[i * ldf + k], Z[i * ldf + k], nrm);
    const float sc = rsqrtf(nrm);
    for (int i = 0; i < n; ++i) Z[i * ldf + k] *= sc;
  }
  __syncthreads();

  // classical Gram-Schmidt, twice, against the earlier members of the eigenvalue's group
  for (int k = 1; k < n; ++k) {
    const int g0 = sm.grp[k];
    if (g0 == k) continue;   // uniform
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = g0 + warp; j < k; j += kEsWarps) {
        float s = 0.f;
        for (int i = lane; i < n; i += 32) s = fmaf(Z[i * ldf + j], Z[i * ldf + k], s);
        s = wsum_f(s);
        if (lane == 0) sm.p[j] = s;
      }
      __syncthreads();
      if (t < n) {
        float zi = Z[t * ldf + k];
        for (int j = g0; j < k; ++j) zi = fmaf(-sm.p[j], Z[t * ldf + j], zi);
        Z[t * ldf + k] = zi;
      }
      __syncthreads();
    }
    float s = 0.f;
    for (int i = lane; i < n; i += 32) s = fmaf(Z[i * ldf + k], Z[i * ldf + k], s);
    s = wsum_f(s);
    __syncthreads();
    if (t < n) Z[t * ldf + k] *= rsqrtf(s);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// The kernel: one cluster of kEsCl CTAs
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kEsThreads, 1)
    eig_small_kernel(int n, const double* __restrict__ Hg, int ldh, double* __restrict__ D,
                     double* __restrict__ Y, int ldy, EsCtl* ctl) {
  extern __shared__ __align__(16) unsigned char es_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int me = (int)cl.block_rank();
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int ld = es_ld(n);
  const EsSmem sm = es_smem(es_raw, n);

  // H (upper triangle, symmetrised) and ||H||_F
  double ss = 0.0;
  for (int idx = t; idx < n * n; idx += kEsThreads) {
    const int i = idx / n, j = idx - i * n;
    const double h = i <= j ? Hg[(size_t)i * ldh + j] : Hg[(size_t)j * ldh + i];
    sm.H[i * ld + j] = h;
    ss = fma(h, h, ss);
  }
  ss = es_block_sum(ss, sm.red);
  const double hnorm = sqrt(ss);
  const int mown = me < n ? (n - me + kEsCl - 1) / kEsCl : 0;
  if (!(hnorm <= DBL_MAX)) {   // non-finite: the Jacobi kernel reports it
    if (me == 0 && t == 0) {
      ctl->run_jacobi = 1;
      ctl->iters = 0;
    }
    return;
  }
  if (n == 1 || hnorm == 0.0) {   // diagonal: D = diag(H) (ascending), Y = permutation
    for (int jj = 0; jj < mown; ++jj) {
      const int j = me + kEsCl * jj;
      const double dj = sm.H[j * ld + j];
      int rk = 0;
      for (int i = 0; i < n; ++i) {
        const double di = sm.H[i * ld + i];
        rk += (di < dj) || (di == dj && i < j);
      }
      if (t == 0) D[rk] = dj;
      for (int i = t; i < n; i += kEsThreads) Y[(size_t)i * ldy + rk] = i == j ? 1.0 : 0.0;
    }
    if (me == 0 && t == 0) {
      ctl->run_jacobi = 0;
      ctl->iters = 0;
    }
    return;
  }

  // every CTA has started (its shared memory exists) before the first remote write
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
  es_float32_phase(sm, n, ldexp(1.0, -ilogb(hnorm)));
  asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
  // X = P_0 P_1 ... P_{n-3} Z for the own columns, a warp per column, pushed to every CTA's X
  // (X is not a float32 work area)
  if (warp < mown) {
    const int c = me + kEsCl * warp, ldf = ld;
    float* Z = sm.Z;
    for (int j = n - 3; j >= 0; --j) {
      const float tau = sm.tau[j];
      if (tau == 0.f) continue;
      const int r = n - j - 1;
      const float* v = sm.V + j * ldf;
      const float z0 = lane < r ? Z[(j + 1 + lane) * ldf + c] : 0.f;
      const float z1 = lane + 32 < r ? Z[(j + 1 + lane + 32) * ldf + c] : 0.f;
      float sv = lane < r ? v[lane] * z0 : 0.f;
      if (lane + 32 < r) sv = fmaf(v[lane + 32], z1, sv);
      sv = tau * wsum_f(sv);
      if (lane < r) Z[(j + 1 + lane) * ldf + c] = fmaf(-v[lane], sv, z0);
      if (lane + 32 < r) Z[(j + 1 + lane + 32) * ldf + c] = fmaf(-v[lane + 32], sv, z1);
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const double x = (double)Z[i * ldf + c];
#pragma unroll 4
      for (int cc = 0; cc < kEsCl; ++cc) cl.map_shared_rank(sm.X, cc)[i * ld + c] = x;
    }
  }
  cl.sync();

  double* Xc = sm.X;
  double* Xo = sm.Xn;
  double emax = 0.0, cpl = 0.0;
  int it = 0;
  for (;;) {
    // own columns j = me + kEsCl jj: P = H X, then S = X^T P and G = X^T X
    for (int o = t; o < n * mown; o += kEsThreads) {
      const int jj = o / n, i = o - jj * n, j = me + kEsCl * jj;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int k = 0;
      for (; k + 3 < n; k += 4) {
        a0 = fma(sm.H[i * ld + k], Xc[k * ld + j], a0);
        a1 = fma(sm.H[i * ld + k + 1], Xc[(k + 1) * ld + j], a1);
        a2 = fma(sm.H[i * ld + k + 2], Xc[(k + 2) * ld + j], a2);
        a3 = fma(sm.H[i * ld + k + 3], Xc[(k + 3) * ld + j], a3);
      }
      for (; k < n; ++k) a0 = fma(sm.H[i * ld + k], Xc[k * ld + j], a0);
      sm.P[jj * n + i] = (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
    for (int o = t; o < 2 * n * mown; o += kEsThreads) {
      const bool gram = o >= n * mown;
      const int oo = gram ? o - n * mown : o;
      const int jj = oo / n, i = oo - jj * n, j = me + kEsCl * jj;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int k = 0;
      if (gram) {
        for (; k + 3 < n; k += 4) {
          a0 = fma(Xc[k * ld + i], Xc[k * ld + j], a0);
          a1 = fma(Xc[(k + 1) * ld + i], Xc[(k + 1) * ld + j], a1);
          a2 = fma(Xc[(k + 2) * ld + i], Xc[(k + 2) * ld + j], a2);
          a3 = fma(Xc[(k + 3) * ld + i], Xc[(k + 3) * ld + j], a3);
        }
        for (; k < n; ++k) a0 = fma(Xc[k * ld + i], Xc[k * ld + j], a0);
        sm.G[jj * n + i] = (a0 + a1) + (a2 + a3);
      } else {
        const double* pc = sm.P + jj * n;
        for (; k + 3 < n; k += 4) {
          a0 = fma(Xc[k * ld + i], pc[k], a0);
          a1 = fma(Xc[(k + 1) * ld + i], pc[k + 1], a1);
          a2 = fma(Xc[(k + 2) * ld + i], pc[k + 2], a2);
          a3 = fma(Xc[(k + 3) * ld + i], pc[k + 3], a3);
        }
        for (; k < n; ++k) a0 = fma(Xc[k * ld + i], pc[k], a0);
        sm.S[jj * n + i] = (a0 + a1) + (a2 + a3);
      }
    }
    __syncthreads();
    // Rayleigh quotients of the own columns, their parts of ||S - diag(lam)||_F^2, ||R||_F^2
    if (warp < mown) {
      const int jj = warp, j = me + kEsCl * jj;
      const double lj = sm.S[jj * n + j] / sm.G[jj * n + j];
      double ps = 0.0, pr = 0.0;
      for (int i = lane; i < n; i += 32) {
        const double ds = sm.S[jj * n + i] - (i == j ? lj : 0.0);
        const double dr = (i == j ? 1.0 : 0.0) - sm.G[jj * n + i];
        ps = fma(ds, ds, ps);
        pr = fma(dr, dr, pr);
      }
      ps = wsum_d(ps);
      pr = wsum_d(pr);
      if (lane == 0) {
        sm.own[jj] = lj;
        sm.own[kEsMaxOwn + jj] = ps;
        sm.own[2 * kEsMaxOwn + jj] = pr;
      }
    }
    __syncthreads();
    if (t < kEsCl) {
      double ps = 0.0, pr = 0.0;
      for (int jj = 0; jj < mown; ++jj) {
        ps += sm.own[kEsMaxOwn + jj];
        pr += sm.own[2 * kEsMaxOwn + jj];
      }
      double* rl = cl.map_shared_rank(sm.lam, t);
      for (int jj = 0; jj < mown; ++jj) rl[me + kEsCl * jj] = sm.own[jj];
      cl.map_shared_rank(sm.sS, t)[me] = ps;
      cl.map_shared_rank(sm.sR, t)[me] = pr;
    }
    cl.sync();
    if (warp == 0) {   // delta = 2 (||S - diag(lam)||_F + ||H||_F ||R||_F), fixed order
      double a = lane < kEsCl ? sm.sS[lane] : 0.0, b = lane < kEsCl ? sm.sR[lane] : 0.0;
#pragma unroll
      for (int o = kEsCl / 2; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
      if (lane == 0) sm.red[kEsWarps] = 2.0 * (sqrt(a) + hnorm * sqrt(b));
    }
    __syncthreads();
    const double delta = sm.red[kEsWarps];
    // E: column j's entries i <= j from the formula, the mirrored E_ji = r_ij - E_ij
    double emx = 0.0, cmx = 0.0;
    for (int o = t; o < n * mown; o += kEsThreads) {
      const int jj = o / n, i = o - jj * n, j = me + kEsCl * jj;
      if (i > j) continue;
      const double lj = sm.lam[j];
      double eij, eji;
      if (i == j) {
        eij = 0.5 * (1.0 - sm.G[jj * n + j]);
        eji = eij;
      } else {
        const double rij = -sm.G[jj * n + i], sij = sm.S[jj * n + i];
        const double gap = lj - sm.lam[i];
        if (fabs(gap) > delta) {
          eij = fma(lj, rij, sij) / gap;
        } else {
          eij = 0.5 * rij;
          cmx = nanmax(cmx, fabs(sij));
        }
        eji = rij - eij;
      }
      emx = nanmax(emx, nanmax(fabs(eij), fabs(eji)));
#pragma unroll 4
      for (int c = 0; c < kEsCl; ++c) {
        double* re = cl.map_shared_rank(sm.E, c);
        re[i * ld + j] = eij;
        re[j * ld + i] = eji;
      }
    }
    emx = wmax_d(emx);
    cmx = wmax_d(cmx);
    if (lane == 0) {
      sm.red[warp] = emx;
      sm.red[kEsWarps + 1 + warp] = cmx;
    }
    __syncthreads();
    if (warp == 0) {
      double a = lane < kEsWarps ? sm.red[lane] : 0.0;
      double b = lane < kEsWarps ? sm.red[kEsWarps + 1 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a = nanmax(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = nanmax(b, __shfl_xor_sync(0xffffffffu, b, o));
      }
      if (lane < kEsCl) {
        cl.map_shared_rank(sm.sE, lane)[me] = a;
        cl.map_shared_rank(sm.sC, lane)[me] = b;
      }
    }
    cl.sync();
    if (warp == 0) {
      double a = lane < kEsCl ? sm.sE[lane] : 0.0, b = lane < kEsCl ? sm.sC[lane] : 0.0;
#pragma unroll
      for (int o = kEsCl / 2; o > 0; o >>= 1) {
        a = nanmax(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = nanmax(b, __shfl_xor_sync(0xffffffffu, b, o));
      }
      if (lane == 0) {
        sm.red[0] = a;
        sm.red[1] = b;
      }
    }
    __syncthreads();
    emax = sm.red[0];
    cpl = sm.red[1];
    const bool last = !(emax > kEsStop) || it + 1 == kEsMaxIt;
    // X' = X + X E, own columns, pushed to every CTA
    for (int o = t; o < n * mown; o += kEsThreads) {
      const int jj = o / n, i = o - jj * n, j = me + kEsCl * jj;
      double a0 = Xc[i * ld + j], a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int k = 0;
      for (; k + 3 < n; k += 4) {
        a0 = fma(Xc[i * ld + k], sm.E[k * ld + j], a0);
        a1 = fma(Xc[i * ld + k + 1], sm.E[(k + 1) * ld + j], a1);
        a2 = fma(Xc[i * ld + k + 2], sm.E[(k + 2) * ld + j], a2);
        a3 = fma(Xc[i * ld + k + 3], sm.E[(k + 3) * ld + j], a3);
      }
      for (; k < n; ++k) a0 = fma(Xc[i * ld + k], sm.E[k * ld + j], a0);
      const double x = (a0 + a1) + (a2 + a3);
#pragma unroll 4
      for (int c = 0; c < kEsCl; ++c) cl.map_shared_rank(Xo, c)[i * ld + j] = x;
    }
    cl.sync();
    double* sw = Xc;
    Xc = Xo;
    Xo = sw;
    ++it;
    if (last) break;
  }

  // ascending order (ties by index); own columns out
  for (int jj = 0; jj < mown; ++jj) {
    const int j = me + kEsCl * jj;
    const double lj = sm.lam[j];
    int rk = 0;
    for (int i = 0; i < n; ++i) {
      const double li = sm.lam[i];
      rk += (li < lj) || (li == lj && i < j);
    }
    if (t == 0 && rk < n) D[rk] = lj;
    for (int i = t; i < n && rk < n; i += kEsThreads) Y[(size_t)i * ldy + rk] = Xc[i * ld + j];
  }
  if (me == 0 && t == 0) {
    const bool ok = emax <= kEsAccept && cpl <= kEsCouple * n * hnorm;
    ctl->run_jacobi = ok ? 0 : 1;
    ctl->iters = it;
  }
}

int es_cluster_ok() {
  // decided once, at the first call (for the largest shared memory, n = kEsMaxN)
  static const int ok = []() {
    const size_t smem = es_smem_bytes(kEsMaxN);
    int v = 0;
    if (cudaFuncSetAttribute(eig_small_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1) == cudaSuccess &&
        cudaFuncSetAttribute(eig_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(kEsCl, 1, 1);
      cfg.blockDim = dim3(kEsThreads, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = kEsCl;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, eig_small_kernel, &cfg) == cudaSuccess &&
          clusters >= 1)
        v = 1;
    }
    cudaGetLastError();
    return v;
  }();
  return ok;
}

}  // namespace

size_t eig_small_work_doubles() { return 8; }

bool eig_small_available() { return es_cluster_ok() != 0; }

cudaError_t launch_eig_small(cudaStream_t st, int n, const double* H, int ldh, double* D,
                             double* Y, int ldy, double* work, int** run_jacobi) {
  *run_jacobi = nullptr;
  if (n < 1 || n > kEsMaxN) return cudaErrorInvalidValue;
  if (!es_cluster_ok()) return cudaErrorNotSupported;
  EsCtl* ctl = reinterpret_cast<EsCtl*>(work);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kEsCl, 1, 1);
  cfg.blockDim = dim3(kEsThreads, 1, 1);
  cfg.dynamicSmemBytes = es_smem_bytes(n);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kEsCl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  note_launch();
  cudaError_t e = cudaLaunchKernelEx(&cfg, eig_small_kernel, n, H, ldh, D, Y, ldy, ctl);
  if (e != cudaSuccess) return e;
  *run_jacobi = &ctl->run_jacobi;
  return cudaSuccess;
}

}  // namespace bchdav
