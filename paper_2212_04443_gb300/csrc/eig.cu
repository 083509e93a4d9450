// Step 9 of Algorithm 2: H Y = Y D for the small symmetric Rayleigh-quotient
// matrix H (n <= act_max), in float64, on the device.
//
// Householder reduction to tridiagonal form (P_k = I - 2 v v^T, applied as
// A <- A - 2 (v w^T + w v^T) with w = A v - (v^T A v) v), backward accumulation
// of Q = P_0 ... P_{n-3}, then the implicitly shifted QL iteration on the
// tridiagonal matrix (Bowdler, Martin, Reinsch, Wilkinson 1968) with each
// sweep's plane rotations recorded by one thread and applied to the rows of
// (QZ)^T by all threads in parallel.  Eigenvalues are returned ascending.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace bchdav {

constexpr int kEigThreads = 1024;

__device__ __forceinline__ double block_sum(double v, double* s_red) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (t == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_red[w];
    s_red[32] = s;
  }
  __syncthreads();
  return s_red[32];
}

__global__ void __launch_bounds__(kEigThreads) eigh_kernel(int n, const double* __restrict__ H,
                                                           int ldh, double* __restrict__ Dout,
                                                           double* __restrict__ Y, int ldy,
                                                           double* __restrict__ work,
                                                           int* __restrict__ status) {
  __shared__ double s_red[33];
  __shared__ double s_scal[4];
  __shared__ int s_int[4];
  extern __shared__ double sdyn[];
  double* d = sdyn;
  double* e = d + n;
  double* cs = e + n;
  double* sn = cs + n;
  double* pv = sn + n;
  int* rank = reinterpret_cast<int*>(pv + n);
  double* A = work;                      // n x n, row-major
  double* Vh = A + (size_t)n * n;        // Householder vectors, row k = v_k
  double* Zt = Vh + (size_t)n * n;       // row j = current eigenvector j
  const int t = threadIdx.x;
  const int T = blockDim.x;
  const int lane = t & 31, warp = t >> 5, nwarps = T >> 5;
  const double eps = 2.220446049250313e-16;

  for (long long idx = t; idx < (long long)n * n; idx += T) {
    int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
    A[idx] = (i <= j) ? H[(size_t)i * ldh + j] : H[(size_t)j * ldh + i];
    Vh[idx] = 0.0;
  }
  __syncthreads();

  // ---- Householder tridiagonalisation
  for (int k = 0; k + 2 < n; ++k) {
    double loc = 0.0;
    for (int i = k + 1 + t; i < n; i += T) {
      double x = A[(size_t)i * n + k];
      loc = fma(x, x, loc);
    }
    double s = block_sum(loc, s_red);
    if (t == 0) {
      double x0 = A[(size_t)(k + 1) * n + k];
      double nx = sqrt(s);
      double alpha = (x0 > 0.0) ? -nx : nx;
      double v0 = x0 - alpha;
      double vn2 = s - x0 * x0 + v0 * v0;
      s_scal[0] = alpha;
      s_scal[1] = (nx > 0.0 && vn2 > 0.0) ? 1.0 / sqrt(vn2) : 0.0;
      s_scal[2] = v0;
    }
    __syncthreads();
    const double inv = s_scal[1];
    if (inv == 0.0) {
      if (t == 0) e[k] = 0.0;
      __syncthreads();
      continue;
    }
    double* v = Vh + (size_t)k * n;
    for (int i = k + 1 + t; i < n; i += T)
      v[i] = (i == k + 1 ? s_scal[2] : A[(size_t)i * n + k]) * inv;
    __syncthreads();
    // p = A22 v (A symmetric: read columns so that consecutive threads are contiguous)
    for (int i = k + 1 + t; i < n; i += T) {
      double p = 0.0;
      for (int j = k + 1; j < n; ++j) p = fma(A[(size_t)j * n + i], v[j], p);
      pv[i] = p;
    }
    __syncthreads();
    loc = 0.0;
    for (int i = k + 1 + t; i < n; i += T) loc = fma(v[i], pv[i], loc);
    double K = block_sum(loc, s_red);
    for (int i = k + 1 + t; i < n; i += T) pv[i] = pv[i] - K * v[i];   // w
    __syncthreads();
    const int m = n - k - 1;
    for (long long idx = t; idx < (long long)m * m; idx += T) {
      int i = k + 1 + (int)(idx / m), j = k + 1 + (int)(idx % m);
      A[(size_t)i * n + j] -= 2.0 * (v[i] * pv[j] + pv[i] * v[j]);
    }
    if (t == 0) e[k] = s_scal[0];
    __syncthreads();
  }
  for (int i = t; i < n; i += T) d[i] = A[(size_t)i * n + i];
  if (t == 0) {
    if (n >= 2) e[n - 2] = A[(size_t)(n - 1) * n + (n - 2)];
    e[n - 1] = 0.0;
  }
  // ---- Q = P_0 ... P_{n-3} (backward accumulation), stored transposed in Zt
  for (long long idx = t; idx < (long long)n * n; idx += T) {
    int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
    Zt[idx] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = n - 3; k >= 0; --k) {
    const double* v = Vh + (size_t)k * n;
    for (int c = k + 1 + warp; c < n; c += nwarps) {
      double* z = Zt + (size_t)c * n;
      double sc = 0.0;
      for (int r = k + 1 + lane; r < n; r += 32) sc = fma(v[r], z[r], sc);
      for (int o = 16; o > 0; o >>= 1) sc += __shfl_xor_sync(0xffffffffu, sc, o);
      for (int r = k + 1 + lane; r < n; r += 32) z[r] = fma(-2.0 * sc, v[r], z[r]);
    }
    __syncthreads();
  }
  // ---- implicit QL on (d, e)
  if (t == 0) s_int[3] = 0;
  __syncthreads();
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      if (t == 0) {
        int m = l;
        for (; m < n - 1; ++m) {
          double dd = fabs(d[m]) + fabs(d[m + 1]);
          if (fabs(e[m]) <= eps * dd) break;
        }
        s_int[0] = m;
        s_int[1] = l;   // lowest rotation index applied this sweep
        s_int[2] = 0;   // 1: underflow restart
        if (m != l) {
          if (iter >= 60) {
            s_int[3] = 1;
            s_int[0] = l;   // give up on this eigenvalue
          } else {
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = m - 1;
            for (; i >= l; --i) {
              double f = s * e[i];
              double bb = c * e[i];
              r = hypot(f, g);
              e[i + 1] = r;
              if (r == 0.0) {
                d[i + 1] -= p;
                e[m] = 0.0;
                break;
              }
              s = f / r;
              c = g / r;
              g = d[i + 1] - p;
              r = (d[i] - g) * s + 2.0 * c * bb;
              p = s * r;
              d[i + 1] = g + p;
              g = c * r - bb;
              cs[i] = c;
              sn[i] = s;
            }
            if (i >= l) {
              s_int[1] = i + 1;
              s_int[2] = 1;
            } else {
              d[l] -= p;
              e[l] = g;
              e[m] = 0.0;
            }
          }
        }
      }
      __syncthreads();
      const int m = s_int[0];
      if (m == l) break;
      const int lo = s_int[1];
      // apply the rotations (i, i+1) for i = m-1 down to lo to the rows of Zt
      for (int r = t; r < n; r += T) {
        for (int i = m - 1; i >= lo; --i) {
          double c = cs[i], s = sn[i];
          double zi = Zt[(size_t)i * n + r];
          double f = Zt[(size_t)(i + 1) * n + r];
          Zt[(size_t)(i + 1) * n + r] = fma(s, zi, c * f);
          Zt[(size_t)i * n + r] = fma(c, zi, -s * f);
        }
      }
      __syncthreads();
    }
  }
  // ---- ascending order (stable ranks), output
  for (int i = t; i < n; i += T) {
    int rk = 0;
    double di = d[i];
    for (int j = 0; j < n; ++j) {
      double dj = d[j];
      rk += (dj < di) || (dj == di && j < i);
    }
    rank[i] = rk;
  }
  __syncthreads();
  for (int i = t; i < n; i += T) Dout[rank[i]] = d[i];
  for (long long idx = t; idx < (long long)n * n; idx += T) {
    int i = (int)(idx / n), r = (int)(idx - (long long)i * n);   // eigenvector i, entry r
    Y[(size_t)r * ldy + rank[i]] = Zt[idx];
  }
  if (t == 0) *status = s_int[3];
}

size_t eigh_work_doubles(int n) { return (size_t)3 * n * n; }

cudaError_t launch_eigh(cudaStream_t st, int n, const double* H, int ldh, double* D, double* Y,
                        int ldy, double* work, int* status) {
  if (n <= 0) return cudaSuccess;
  if (n > 4096) return cudaErrorInvalidValue;
  size_t smem = (size_t)5 * n * sizeof(double) + (size_t)n * sizeof(int);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(eigh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  eigh_kernel<<<1, kEigThreads, smem, st>>>(n, H, ldh, D, Y, ldy, work, status); note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Multi-SM variant: parallel cyclic Jacobi.
//
// On GB300 a float64 operation has a long latency and one SM retires only 2
// float64 FMA per clock, so the implicit QL recurrence (one long dependent
// chain of divisions and square roots) and any O(n^3) work on a single SM are
// slow.  The two-sided Jacobi method instead rotates n/2 disjoint index pairs
// at once (round-robin "circle" ordering, n - 1 rounds per sweep): every CTA
// computes the same rotations of a round from the current diagonal and pair
// entries (Rutishauser's formulas), then the grid updates the disjoint 2x2
// blocks of A <- J^T A J and the column pairs of V <- V J, and one grid barrier
// ends the round.  Sweeps repeat until the off-diagonal mass is below
// (eps * ||A||_F)^2.  Eigenvalues come out on the diagonal, sorted ascending
// at the end with their columns of V.

constexpr int kJacThreads = 256;
constexpr int kJacPre = 4;   // items per thread whose operands are loaded ahead of the angles
constexpr int kJacMaxSweeps = 40;

struct JacLayout {
  double *A, *V, *red, *ang;
  int* status;
};

__host__ __device__ inline JacLayout jac_layout(double* w, int n) {
  JacLayout L;
  const int np = n + (n & 1);
  L.A = w;
  L.V = L.A + (size_t)np * np;
  L.red = L.V + (size_t)np * np;   // [2][grid] partial sums
  L.ang = L.red + 2 * 4 * kSMs;     // [2][np / 2][3] angle inputs (a_pp, a_qq, a_pq) by round parity
  L.status = reinterpret_cast<int*>(L.ang + 3 * (size_t)np + 8);
  return L;
}

size_t eigh_fast_work_doubles(int n) {
  const size_t np = (size_t)(n + (n & 1));
  return 2 * np * np + 2 * 4 * kSMs + 3 * np + 16;
}

// player at circle position `pos` in round r (n_pad players, player 0 fixed)
__device__ __forceinline__ int jac_player(int pos, int r, int np) {
  return pos == 0 ? 0 : 1 + (pos - 1 + r) % (np - 1);
}
// circle position of player x in round r (inverse of jac_player)
__device__ __forceinline__ int jac_pos(int x, int r, int np) {
  if (x == 0) return 0;
  int t = (x - 1 - r) % (np - 1);
  if (t < 0) t += np - 1;
  return t + 1;
}
// position of a player in the next round: everyone but player 0 moves one place back on the
// circle (position 1 wraps to np - 1)
__device__ __forceinline__ int jac_next_pos(int pos, int np) {
  return pos == 0 ? 0 : (pos == 1 ? np - 1 : pos - 1);
}

// Entry (x, y) of A, just rotated in round r, with next-round positions px, py: if round
// r + 1 needs it to compute a rotation angle (a diagonal entry of one of its pairs, or a
// pair's off-diagonal entry), store it in that round's angle-input slots.  The slots of a
// round are written only in the round before and read only in that round (double buffered by
// parity), so no CTA can read a value that another CTA is rewriting in the same round.
__device__ __forceinline__ void jac_note_next(double* __restrict__ ang, int x, int y, int px,
                                              int py, double v, int r, int np, int wbuf) {
  const int half = np / 2;
  const int kx = px < half ? px : np - 1 - px;
  double* slot = ang + (size_t)wbuf * 3 * half + 3 * kx;
  if (x == y) {
    const int partner = jac_player(np - 1 - px, r + 1, np);
    slot[x < partner ? 0 : 1] = v;
  } else if (x < y && px + py == np - 1) {
    slot[2] = v;
  }
}

__global__ void __launch_bounds__(kJacThreads) jacobi_coop_kernel(int n, const double* __restrict__ H,
                                                                  int ldh, double* __restrict__ work,
                                                                  double* __restrict__ Dout,
                                                                  double* __restrict__ Y, int ldy) {
  cg::grid_group grid = cg::this_grid();
  const int np = n + (n & 1);   // an odd n gets a dummy index n that is never rotated
  const int half = np / 2;
  JacLayout L = jac_layout(work, n);
  extern __shared__ double sj[];
  double* cs = sj;            // half
  double* sn = sj + half;     // half
  int* pp = reinterpret_cast<int*>(sj + 2 * half);   // half
  int* qq = pp + half;                               // half
  int* npp = qq + half;                              // half: next-round position of pp[k]
  int* nqq = npp + half;                             // half: next-round position of qq[k]
  __shared__ double s_red[33];
  __shared__ int s_flag;
  const int t = threadIdx.x;
  const long long gtid = (long long)blockIdx.x * kJacThreads + t;
  const long long gstride = (long long)gridDim.x * kJacThreads;
  double* A = L.A;
  double* V = L.V;
  // A = H (symmetric, upper triangle read), padded row/column zero; V = I
  for (long long idx = gtid; idx < (long long)np * np; idx += gstride) {
    int i = (int)(idx / np), j = (int)(idx - (long long)i * np);
    double a = 0.0;
    if (i < n && j < n) a = (i <= j) ? H[(size_t)i * ldh + j] : H[(size_t)j * ldh + i];
    A[idx] = a;
    V[idx] = (i == j) ? 1.0 : 0.0;
  }
  // angle inputs of round 0, straight from H
  for (long long k = gtid; k < half; k += gstride) {
    int p = jac_player((int)k, 0, np), q = jac_player(np - 1 - (int)k, 0, np);
    if (p > q) {
      const int x = p;
      p = q;
      q = x;
    }
    auto h = [&](int i, int j) {
      return (i < n && j < n) ? ((i <= j) ? H[(size_t)i * ldh + j] : H[(size_t)j * ldh + i]) : 0.0;
    };
    L.ang[3 * k] = h(p, p);
    L.ang[3 * k + 1] = h(q, q);
    L.ang[3 * k + 2] = h(p, q);
  }
  // ||A||_F^2 for the stopping threshold
  double loc = 0.0;
  for (long long idx = gtid; idx < (long long)np * np; idx += gstride) loc = fma(A[idx], A[idx], loc);
  double tot = block_sum(loc, s_red);
  if (t == 0) L.red[blockIdx.x] = tot;
  grid.sync();
  if (t == 0) {
    double sacc = 0.0;
    for (int g = 0; g < (int)gridDim.x; ++g) sacc += L.red[g];
    s_red[32] = sacc;
  }
  __syncthreads();
  const double eps = 2.220446049250313e-16;
  const double thresh = eps * eps * s_red[32];
  int status = 1;
  for (int sweep = 0; sweep < kJacMaxSweeps; ++sweep) {
    for (int r = 0; r < np - 1; ++r) {
      const int rbuf = (int)(((long long)sweep * (np - 1) + r) & 1);   // angle inputs read now
      // The pairs of round r are fixed by r alone, so each thread first loads the entries its
      // (at most kJacPre) items will rotate, then the angles are computed while those loads
      // are in flight; the arithmetic is that of one rotation at a time per entry.
      const long long nblk = (long long)half * half;
      const long long nitems = nblk + (long long)np * half;
      double pre[kJacPre][4];
      int ppre[kJacPre][4];
#pragma unroll
      for (int u = 0; u < kJacPre; ++u) {
        const long long idx = gtid + u * gstride;
        ppre[u][0] = -1;
        if (idx >= nitems) continue;
        if (idx < nblk) {
          const int K = (int)(idx / half), Lb = (int)(idx - (long long)K * half);
          int p1 = jac_player(K, r, np), q1 = jac_player(np - 1 - K, r, np);
          int p2 = jac_player(Lb, r, np), q2 = jac_player(np - 1 - Lb, r, np);
          if (p1 > q1) { const int x = p1; p1 = q1; q1 = x; }
          if (p2 > q2) { const int x = p2; p2 = q2; q2 = x; }
          ppre[u][0] = (int)(p1 * np + p2);
          ppre[u][1] = (int)(p1 * np + q2);
          ppre[u][2] = (int)(q1 * np + p2);
          ppre[u][3] = (int)(q1 * np + q2);
          pre[u][0] = A[ppre[u][0]];
          pre[u][1] = A[ppre[u][1]];
          pre[u][2] = A[ppre[u][2]];
          pre[u][3] = A[ppre[u][3]];
        } else {
          const long long j = idx - nblk;
          const int row = (int)(j / half), K = (int)(j - (long long)row * half);
          int p = jac_player(K, r, np), q = jac_player(np - 1 - K, r, np);
          if (p > q) { const int x = p; p = q; q = x; }
          ppre[u][0] = (int)(row * np + p);
          ppre[u][1] = (int)(row * np + q);
          pre[u][0] = V[ppre[u][0]];
          pre[u][1] = V[ppre[u][1]];
        }
      }
      // rotations of this round, computed identically by every CTA
      for (int k = t; k < half; k += kJacThreads) {
        int p = jac_player(k, r, np), q = jac_player(np - 1 - k, r, np);
        if (p > q) {
          int tmp = p;
          p = q;
          q = tmp;
        }
        pp[k] = p;
        qq[k] = q;
        {
          // positions this round: k holds player(k), np - 1 - k holds the other
          const int pos_p = (p == jac_player(k, r, np)) ? k : np - 1 - k;
          npp[k] = jac_next_pos(pos_p, np);
          nqq[k] = jac_next_pos(np - 1 - pos_p, np);
        }
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double* in = L.ang + (size_t)rbuf * 3 * half + 3 * k;
          const double apq = in[2];
          if (apq != 0.0) {
            const double app = in[0], aqq = in[1];
            const double theta = (aqq - app) / (2.0 * apq);
            const double tt = copysign(1.0, theta) / (fabs(theta) + sqrt(fma(theta, theta, 1.0)));
            c = 1.0 / sqrt(fma(tt, tt, 1.0));
            s = tt * c;
          }
        }
        cs[k] = c;
        sn[k] = s;
      }
      __syncthreads();
      // A <- J^T A J on the 2x2 blocks (K, L); V <- V J on the column pairs
      auto apply = [&](long long idx, double (&x)[4], const int (&off)[4], bool loaded) {
        if (idx < nblk) {
          const int K = (int)(idx / half), Lb = (int)(idx - (long long)K * half);
          const double c1 = cs[K], s1 = sn[K], c2 = cs[Lb], s2 = sn[Lb];
          const int p1 = pp[K], q1 = qq[K], p2 = pp[Lb], q2 = qq[Lb];
          int o[4] = {off[0], off[1], off[2], off[3]};
          if (!loaded) {
            o[0] = p1 * np + p2;
            o[1] = p1 * np + q2;
            o[2] = q1 * np + p2;
            o[3] = q1 * np + q2;
#pragma unroll
            for (int e = 0; e < 4; ++e) x[e] = A[o[e]];
          }
          double z[4] = {x[0], x[1], x[2], x[3]};
          if (!(s1 == 0.0 && s2 == 0.0)) {
            const double x11 = x[0], x12 = x[1], x21 = x[2], x22 = x[3];
            // rows: J1^T X
            const double y11 = c1 * x11 - s1 * x21, y12 = c1 * x12 - s1 * x22;
            const double y21 = s1 * x11 + c1 * x21, y22 = s1 * x12 + c1 * x22;
            // columns: (J1^T X) J2
            z[0] = c2 * y11 - s2 * y12;
            z[1] = s2 * y11 + c2 * y12;
            z[2] = c2 * y21 - s2 * y22;
            z[3] = s2 * y21 + c2 * y22;
            if (K == Lb) z[1] = z[2] = 0.0;   // the pair entry this rotation annihilates
#pragma unroll
            for (int e = 0; e < 4; ++e) A[o[e]] = z[e];
          }
          {
            const int np1 = npp[K], nq1 = nqq[K], np2 = npp[Lb], nq2 = nqq[Lb];
            jac_note_next(L.ang, p1, p2, np1, np2, z[0], r, np, rbuf ^ 1);
            jac_note_next(L.ang, p1, q2, np1, nq2, z[1], r, np, rbuf ^ 1);
            jac_note_next(L.ang, q1, p2, nq1, np2, z[2], r, np, rbuf ^ 1);
            jac_note_next(L.ang, q1, q2, nq1, nq2, z[3], r, np, rbuf ^ 1);
          }
        } else {
          const long long j = idx - nblk;
          const int row = (int)(j / half), K = (int)(j - (long long)row * half);
          const double c = cs[K], s = sn[K];
          if (s == 0.0) return;
          int o0 = off[0], o1 = off[1];
          if (!loaded) {
            o0 = row * np + pp[K];
            o1 = row * np + qq[K];
            x[0] = V[o0];
            x[1] = V[o1];
          }
          const double xp = x[0], xq = x[1];
          V[o0] = c * xp - s * xq;
          V[o1] = s * xp + c * xq;
        }
      };
#pragma unroll
      for (int u = 0; u < kJacPre; ++u) {
        const long long idx = gtid + u * gstride;
        if (idx < nitems) apply(idx, pre[u], ppre[u], true);
      }
      for (long long idx = gtid + kJacPre * gstride; idx < nitems; idx += gstride) {
        double x[4];
        const int off[4] = {0, 0, 0, 0};
        apply(idx, x, off, false);
      }
      grid.sync();
    }
    // off-diagonal mass after the sweep
    loc = 0.0;
    for (long long idx = gtid; idx < (long long)np * np; idx += gstride) {
      int i = (int)(idx / np), j = (int)(idx - (long long)i * np);
      if (i != j) loc = fma(A[idx], A[idx], loc);
    }
    tot = block_sum(loc, s_red);
    if (t == 0) L.red[((sweep + 1) & 1) * 4 * kSMs + blockIdx.x] = tot;
    grid.sync();
    if (t == 0) {
      double sacc = 0.0;
      for (int g = 0; g < (int)gridDim.x; ++g) sacc += L.red[((sweep + 1) & 1) * 4 * kSMs + g];
      s_flag = (sacc <= thresh) ? 1 : 0;
    }
    __syncthreads();
    if (s_flag) {
      status = 0;
      break;
    }
  }
  // ascending order of the diagonal (stable ranks); every CTA writes a share of the output
  for (int i = (int)gtid; i < n; i += (int)gstride) {
    const double di = A[(size_t)i * np + i];
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const double dj = A[(size_t)j * np + j];
      rk += (dj < di) || (dj == di && j < i);
    }
    Dout[rk] = di;
    for (int row = 0; row < n; ++row) Y[(size_t)row * ldy + rk] = V[(size_t)row * np + i];
  }
  if (gtid == 0) *L.status = status;
}

cudaError_t launch_eigh_fast(cudaStream_t st, int n, const double* H, int ldh, double* D, double* Y,
                             int ldy, double* work, int* status, int grid_cap) {
  if (n <= 32) return launch_eigh(st, n, H, ldh, D, Y, ldy, work, status);
  if (n > 1024) return cudaErrorInvalidValue;
  const int np = n + (n & 1);
  const size_t smem = (size_t)(np / 2) * (2 * sizeof(double) + 4 * sizeof(int));
  // one wave of co-resident blocks (thread-safe static initialisation)
  static const int max_blocks = []() {
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_coop_kernel, kJacThreads,
                                                      16 * 1024) != cudaSuccess) {
      cudaGetLastError();
      return 1;
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, per_sm * sms);
  }();
  // enough threads for the largest round (blocks + vector pairs), at most one wave; the
  // items-per-thread target trades grid-barrier cost against per-round work (tunable with
  // BCHDAV_JACOBI_ITEMS)
  static const int items_per_thread = []() {
    const char* env = getenv("BCHDAV_JACOBI_ITEMS");
    return env ? std::max(1, atoi(env)) : 2;
  }();
  long long work_items = (long long)(np / 2) * (np / 2) + (long long)np * (np / 2);
  int grid = ceil_div(work_items, (long long)kJacThreads * items_per_thread);
  if (grid > max_blocks) grid = max_blocks;
  if (grid > 4 * kSMs) grid = 4 * kSMs;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  if (grid < 1) grid = 1;
  JacLayout L = jac_layout(work, n);
  int nn = n, lh = ldh, ly = ldy;
  double* wk = work;
  void* args[] = {&nn, (void*)&H, &lh, &wk, &D, &Y, &ly};
  note_launch();
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)jacobi_coop_kernel, grid, kJacThreads,
                                              args, smem, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(status, L.status, sizeof(int), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of bchdav_eigh.
//
// Some callers cannot allocate device memory at the time they need this
// eigensolver: code running while another runtime owns every byte of device
// memory through its own pool, or a latency-critical path that must not take
// the device-wide synchronisation cudaMalloc and cudaFree can imply.  For them
// the scratch lives in this fixed, file-scope device array, sized for
// n <= kNoAllocMaxN (3 * 128 * 128 doubles for the work area plus one status
// word, about 384 KiB).  Every GPU that loads the library reserves it until the
// process exits.  In host code `g_eigh_scratch` only names a host-side stand-in,
// so its device address is fetched with cudaGetSymbolAddress, once per device,
// with that device current, on the first call made on it; that first call
// should therefore come before any stream capture.  All calls share the array
// and it keeps the last call's contents: the status word is cleared on every
// call, the kernel overwrites the work area before reading it, and calls whose
// work overlaps on the GPU race with one another.
namespace {
constexpr int kNoAllocMaxN = 128;
constexpr size_t kNoAllocWork = (size_t)3 * kNoAllocMaxN * kNoAllocMaxN;
constexpr int kMaxDevices = 64;
__device__ __align__(256) double g_eigh_scratch[kNoAllocWork + 32];
std::mutex g_noalloc_mu;
double* g_noalloc_base[kMaxDevices] = {};
}  // namespace

void set_global_error(const char* msg);

}  // namespace bchdav

extern "C" bchdav_status bchdav_eigh_noalloc(int32_t n, const double* H, int32_t ld_h, double* D,
                                             double* Y, int32_t ld_y, void* cuda_stream) {
  using namespace bchdav;
  if (n < 1 || n > kNoAllocMaxN || ld_h < n || ld_y < n || !H || !D || !Y) {
    set_global_error(n > kNoAllocMaxN
                         ? "eigh_noalloc: n exceeds the fixed scratch (n <= 128)"
                         : "eigh_noalloc: invalid arguments");
    return BCHDAV_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_global_error("eigh_noalloc: no usable current device");
    return BCHDAV_ERR_CUDA;
  }
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_eigh_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        set_global_error("eigh_noalloc: cudaGetSymbolAddress failed");
        return BCHDAV_ERR_CUDA;
      }
      g_noalloc_base[dev] = static_cast<double*>(p);
    }
    base = g_noalloc_base[dev];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int* status = reinterpret_cast<int*>(base + kNoAllocWork);
  int host_status = 0;
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = launch_eigh(st, n, H, ld_h, D, Y, ld_y, base, status);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_global_error("eigh_noalloc: CUDA error");
    return BCHDAV_ERR_CUDA;
  }
  if (host_status != 0) {
    set_global_error("eigh_noalloc: QL iteration did not converge");
    return BCHDAV_ERR_NONFINITE;
  }
  return BCHDAV_OK;
}
