// Step 9 of Algorithm 2: H Y = Y D for the small symmetric Rayleigh-quotient
// matrix H (n <= act_max), in float64, on the device.  launch_eigh_fast picks the
// route (eigs.cu for n <= 64, trd.cu up to 448, the Jacobi kernel below beyond that
// and as the device-gated fallback of both); this file also holds the one-block
// kernel of the allocation-free entry point and of the Lanczos bounds:
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
// (about 1.3 us on GB300, whatever the grid) ends the round.  Sweeps repeat
// until the off-diagonal mass is below (eps * ||A||_F)^2 or a sweep finds
// nothing to rotate.  Eigenvalues come out on the diagonal, sorted ascending
// at the end with their columns of V.

constexpr int kJacThreads = 256;
constexpr int kJacPre = 4;   // items per thread whose operands are loaded ahead of the angles
constexpr int kJacMaxSweeps = 40;

struct JacLayout {
  double *A, *V, *red, *ang;
  int* status;               // 0 converged, 1 sweep limit, 2 a grid barrier gave up
  unsigned* bar;             // arrivals at the grid barrier (zeroed before each launch)
  int* where;                // the barrier that gave up: sweep * 4096 + round (debug)
};

__host__ __device__ inline JacLayout jac_layout(double* w, int n) {
  JacLayout L;
  const int np = n + (n & 1);
  L.A = w;
  L.V = L.A + (size_t)np * np;
  L.red = L.V + (size_t)np * np;   // [2][grid] partial sums
  L.ang = L.red + 2 * 4 * kSMs;     // [2][np / 2][3] angle inputs (a_pp, a_qq, a_pq) by round parity
  L.status = reinterpret_cast<int*>(L.ang + 3 * (size_t)np + 8);
  L.bar = reinterpret_cast<unsigned*>(L.status + 2);
  L.where = L.status + 4;
  return L;
}

static size_t jacobi_work_doubles(int n) {
  const size_t np = (size_t)(n + (n & 1));
  return 2 * np * np + 2 * 4 * kSMs + 3 * np + 16;
}

// the Jacobi area first (its status word is the route's), the small or tridiagonal route's after it
size_t eigh_fast_work_doubles(int n) {
  const size_t small = n <= kEsMaxN ? eig_small_work_doubles() : 0;
  const size_t trd = n > 32 && n <= kTrdMaxN ? trd_work_doubles(n) : 0;
  return jacobi_work_doubles(n) + std::max(small, trd);
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

// A is kept in its upper triangle only (entry (i, j) at min(i, j) * np + max(i, j)): a round
// updates the 2x2 blocks (K, L) with K <= L, half of the float64 work of the full matrix.
//
// A rotation whose pair entry is negligible, a_pq^2 <= eps^2 |a_pp a_qq| (it changes the
// eigenvalues by O(eps) relative and the eigenvectors by O(eps / relative gap)), is not applied.
// Every CTA computes every angle of a round, so all of them see the same decisions: a round
// without a rotation is skipped by all (no update, no barrier), and a sweep without a rotation
// ends the iteration (A is diagonal to working accuracy), as does the off-diagonal mass test.
// After a skipped round the next round reads its angle inputs from A itself, so before it
// updates A it waits at a barrier until every CTA has read them.
// Grid barrier of the cooperative launch with a bounded wait: thread 0 of each CTA adds its
// arrival and polls the count until every CTA of this barrier instance has arrived; after
// kJacSpin polls it gives up, and the CTA stops (status 2) instead of waiting forever.  Reads of
// data other CTAs wrote go through L2 (__ldcg), so nothing stale is served from L1.
constexpr long long kJacSpin = 1LL << 25;

__device__ __forceinline__ bool jac_barrier(unsigned* bar, unsigned target, int* s_abort) {
  __syncthreads();
  if (threadIdx.x == 0 && !*s_abort) {
    __threadfence();
    atomicAdd(bar, 1u);
    long long i = 0;
    while (*reinterpret_cast<volatile unsigned*>(bar) < target) {
      if (++i > kJacSpin) {
        *s_abort = 1;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return !*s_abort;
}

__device__ __forceinline__ int jac_ut(int i, int j, int np) {
  return i < j ? i * np + j : j * np + i;
}

// run_if (optional): the kernel does nothing unless *run_if is nonzero (the tridiagonal route
// ran before it and asks for its result to be replaced); every CTA reads the same word.
__global__ void __launch_bounds__(kJacThreads) jacobi_coop_kernel(int n, const double* __restrict__ H,
                                                                  int ldh, double* __restrict__ work,
                                                                  double* __restrict__ Dout,
                                                                  double* __restrict__ Y, int ldy,
                                                                  const int* __restrict__ run_if) {
  if (run_if && *reinterpret_cast<const volatile int*>(run_if) == 0) return;
  const int np = n + (n & 1);   // an odd n gets a dummy index n that is never rotated
  const int half = np / 2;
  JacLayout L = jac_layout(work, n);
  __shared__ int s_abort;
  if (threadIdx.x == 0) s_abort = 0;
  unsigned bar_target = 0;
  int where = -1;
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
  // A = H (upper triangle read), padded row/column zero; V = I
  for (long long idx = gtid; idx < (long long)np * np; idx += gstride) {
    int i = (int)(idx / np), j = (int)(idx - (long long)i * np);
    double a = 0.0;
    if (i < n && j < n) a = (i <= j) ? H[(size_t)i * ldh + j] : H[(size_t)j * ldh + i];
    A[idx] = a;
    V[idx] = (i == j) ? 1.0 : 0.0;
  }
  // ||A||_F^2 for the stopping threshold
  double loc = 0.0;
  for (long long idx = gtid; idx < (long long)np * np; idx += gstride) loc = fma(A[idx], A[idx], loc);
  double tot = block_sum(loc, s_red);
  if (t == 0) L.red[blockIdx.x] = tot;
  bar_target += gridDim.x;
  jac_barrier(L.bar, bar_target, &s_abort);
  if (t == 0) {
    double sacc = 0.0;
    for (int g = 0; g < (int)gridDim.x; ++g) sacc += __ldcg(L.red + g);
    s_red[32] = sacc;
  }
  __syncthreads();
  const double eps = 2.220446049250313e-16;
  const double thresh = eps * eps * s_red[32];
  int status = 1;
  // where the angle inputs of the next round are: A itself (after a skipped round, and at the
  // start), or the slots of buffer rb written by the round before
  bool from_A = true;
  int rb = 0;
  const long long nblk = (long long)half * (half + 1) / 2;   // blocks K <= L
  const long long nitems = nblk + (long long)np * half;
  for (int sweep = 0; sweep < kJacMaxSweeps && !s_abort; ++sweep) {
    bool sweep_rotated = false;
    for (int r = 0; r < np - 1 && !s_abort; ++r) {
      const int wb = from_A ? rb : rb ^ 1;   // buffer this round's notes go to
      // block (K, L), K <= L, of item idx < nblk (L-major)
      auto block_of = [&](long long idx, int& K, int& Lb) {
        int l = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
        while ((long long)l * (l + 1) / 2 > idx) --l;
        while ((long long)(l + 1) * (l + 2) / 2 <= idx) ++l;
        Lb = l;
        K = (int)(idx - (long long)l * (l + 1) / 2);
      };
      auto ordered_pair = [&](int k, int& p, int& q) {
        p = jac_player(k, r, np);
        q = jac_player(np - 1 - k, r, np);
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
      };
      // The pairs of round r are fixed by r alone, so each thread first loads the entries its
      // (at most kJacPre) items will rotate, then the angles are computed while those loads
      // are in flight; the arithmetic is that of one rotation at a time per entry.
      double pre[kJacPre][4];
      int ppre[kJacPre][4];
#pragma unroll
      for (int u = 0; u < kJacPre; ++u) {
        const long long idx = gtid + u * gstride;
        ppre[u][0] = -1;
        if (idx >= nitems) continue;
        if (idx < nblk) {
          int K, Lb, p1, q1, p2, q2;
          block_of(idx, K, Lb);
          ordered_pair(K, p1, q1);
          ordered_pair(Lb, p2, q2);
          ppre[u][0] = jac_ut(p1, p2, np);
          ppre[u][1] = jac_ut(p1, q2, np);
          ppre[u][2] = jac_ut(q1, p2, np);
          ppre[u][3] = jac_ut(q1, q2, np);
          pre[u][0] = __ldcg(A + ppre[u][0]);
          pre[u][1] = __ldcg(A + ppre[u][1]);
          pre[u][2] = __ldcg(A + ppre[u][2]);
          pre[u][3] = __ldcg(A + ppre[u][3]);
        } else {
          const long long j = idx - nblk;
          const int row = (int)(j / half), K = (int)(j - (long long)row * half);
          int p, q;
          ordered_pair(K, p, q);
          ppre[u][0] = (int)(row * np + p);
          ppre[u][1] = (int)(row * np + q);
          pre[u][0] = __ldcg(V + ppre[u][0]);
          pre[u][1] = __ldcg(V + ppre[u][1]);
        }
      }
      // rotations of this round, computed identically by every CTA
      int mine = 0;
      for (int k = t; k < half; k += kJacThreads) {
        int p, q;
        ordered_pair(k, p, q);
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
          double app, aqq, apq;
          if (from_A) {
            app = __ldcg(A + (size_t)p * np + p);
            aqq = __ldcg(A + (size_t)q * np + q);
            apq = __ldcg(A + (size_t)p * np + q);
          } else {
            const double* in = L.ang + (size_t)rb * 3 * half + 3 * k;
            app = __ldcg(in);
            aqq = __ldcg(in + 1);
            apq = __ldcg(in + 2);
          }
          if (apq != 0.0 && apq * apq > eps * eps * fabs(app * aqq)) {
            const double theta = (aqq - app) / (2.0 * apq);
            const double tt = copysign(1.0, theta) / (fabs(theta) + sqrt(fma(theta, theta, 1.0)));
            c = 1.0 / sqrt(fma(tt, tt, 1.0));
            s = tt * c;
            mine = 1;
          }
        }
        cs[k] = c;
        sn[k] = s;
      }
      if (!__syncthreads_or(mine)) {   // the same in every CTA: nothing rotates this round
        from_A = true;
        continue;
      }
      sweep_rotated = true;
      // A round that read its angle inputs from A must not update A before every CTA has read
      // them (a faster CTA would otherwise overwrite entries a slower one has yet to read)
      if (from_A) {
        bar_target += gridDim.x;
        if (!jac_barrier(L.bar, bar_target, &s_abort)) {
          where = sweep * 4096 + r;
          break;
        }
      }
      // A <- J^T A J on the upper-triangle 2x2 blocks (K, L); V <- V J on the column pairs
      auto apply = [&](long long idx, double (&x)[4], const int (&off)[4], bool loaded) {
        if (idx < nblk) {
          int K, Lb;
          block_of(idx, K, Lb);
          const double c1 = cs[K], s1 = sn[K], c2 = cs[Lb], s2 = sn[Lb];
          const int p1 = pp[K], q1 = qq[K], p2 = pp[Lb], q2 = qq[Lb];
          int o[4] = {off[0], off[1], off[2], off[3]};
          if (!loaded) {
            o[0] = jac_ut(p1, p2, np);
            o[1] = jac_ut(p1, q2, np);
            o[2] = jac_ut(q1, p2, np);
            o[3] = jac_ut(q1, q2, np);
#pragma unroll
            for (int e = 0; e < 4; ++e) x[e] = __ldcg(A + o[e]);
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
            const int xs[4] = {p1, p1, q1, q1}, ys[4] = {p2, q2, p2, q2};
            const int pxs[4] = {np1, np1, nq1, nq1}, pys[4] = {np2, nq2, np2, nq2};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (xs[e] <= ys[e])
                jac_note_next(L.ang, xs[e], ys[e], pxs[e], pys[e], z[e], r, np, wb);
              else
                jac_note_next(L.ang, ys[e], xs[e], pys[e], pxs[e], z[e], r, np, wb);
            }
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
            x[0] = __ldcg(V + o0);
            x[1] = __ldcg(V + o1);
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
      bar_target += gridDim.x;
      if (!jac_barrier(L.bar, bar_target, &s_abort)) {
        where = sweep * 4096 + r;
        break;
      }
      from_A = false;
      rb = wb;
    }
    if (s_abort) break;
    if (!sweep_rotated) {   // the same in every CTA
      status = 0;
      break;
    }
    // off-diagonal mass after the sweep (upper triangle, counted twice)
    loc = 0.0;
    for (long long idx = gtid; idx < (long long)np * np; idx += gstride) {
      int i = (int)(idx / np), j = (int)(idx - (long long)i * np);
      if (i < j) {
        const double a = __ldcg(A + idx);
        loc = fma(2.0 * a, a, loc);
      }
    }
    tot = block_sum(loc, s_red);
    if (t == 0) L.red[((sweep + 1) & 1) * 4 * kSMs + blockIdx.x] = tot;
    bar_target += gridDim.x;
    if (!jac_barrier(L.bar, bar_target, &s_abort)) {
      where = sweep * 4096 + 4095;
      break;
    }
    if (t == 0) {
      double sacc = 0.0;
      for (int g = 0; g < (int)gridDim.x; ++g)
        sacc += __ldcg(L.red + ((sweep + 1) & 1) * 4 * kSMs + g);
      s_flag = (sacc <= thresh) ? 1 : 0;
    }
    __syncthreads();
    if (s_flag) {
      status = 0;
      break;
    }
  }
  if (s_abort) {
    // a barrier gave up: report it and write nothing (the other CTAs stop at theirs)
    if (threadIdx.x == 0) {
      atomicExch(L.status, 2);
      if (where >= 0) atomicExch(L.where, where);
    }
    return;
  }
  // ascending order of the diagonal (stable ranks); every CTA writes a share of the output
  for (int i = (int)gtid; i < n; i += (int)gstride) {
    const double di = __ldcg(A + (size_t)i * np + i);
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const double dj = __ldcg(A + (size_t)j * np + j);
      rk += (dj < di) || (dj == di && j < i);
    }
    Dout[rk] = di;
    for (int row = 0; row < n; ++row) Y[(size_t)row * ldy + rk] = __ldcg(V + (size_t)row * np + i);
  }
  if (gtid == 0) atomicMax(L.status, status);
}

cudaError_t launch_eigh_fast(cudaStream_t st, int n, const double* H, int ldh, double* D, double* Y,
                             int ldy, double* work, int* status, int grid_cap, cudaStream_t aux,
                             cudaEvent_t ev1, cudaEvent_t ev2) {
  const bool small = n <= kEsMaxN && eig_small_available();
  if (n <= 32 && !small) return launch_eigh(st, n, H, ldh, D, Y, ldy, work, status);
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
  // a round's items (upper-triangle blocks + vector pairs) over at most one block per SM: the
  // barrier costs the same for any grid, the float64 work shrinks with every SM added; an
  // items-per-thread floor (BCHDAV_JACOBI_ITEMS, default 1) keeps small problems on fewer SMs
  static const int items_per_thread = []() {
    const char* env = getenv("BCHDAV_JACOBI_ITEMS");
    return env ? std::max(1, atoi(env)) : 1;
  }();
  static const int sms = []() {
    int dev = 0, v = kSMs;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : kSMs;
  }();
  const long long work_items =
      (long long)(np / 2) * (np / 2 + 1) / 2 + (long long)np * (np / 2);
  int grid = ceil_div(work_items, (long long)kJacThreads * items_per_thread);
  if (grid > max_blocks) grid = max_blocks;
  if (grid > sms) grid = sms;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  if (grid < 1) grid = 1;
  JacLayout L = jac_layout(work, n);
  cudaError_t e0 = cudaMemsetAsync(L.status, 0, 6 * sizeof(int), st);   // status, bar, where
  if (e0 != cudaSuccess) return e0;
  // the small or the tridiagonal route where the device runs it; the Jacobi kernel then runs
  // only when the route flags its result (for the small route: the refinement not converged or
  // a cluster left coupled; for the tridiagonal one: a tight cluster too wide, orthogonality out
  // of reach; for both: a non-finite H)
  int* run_if = nullptr;
  if (small) {
    cudaError_t es = launch_eig_small(st, n, H, ldh, D, Y, ldy, work + jacobi_work_doubles(n),
                                      &run_if);
    if (es != cudaSuccess) return es;
  } else if (n <= kTrdMaxN) {
    cudaError_t et = launch_trd_eigh(st, n, H, ldh, D, Y, ldy, work + jacobi_work_doubles(n),
                                     &run_if, aux, ev1, ev2);
    if (et == cudaErrorNotSupported) {
      run_if = nullptr;
    } else if (et != cudaSuccess) {
      return et;
    }
  }
  int nn = n, lh = ldh, ly = ldy;
  double* wk = work;
  const int* ri = run_if;
  void* args[] = {&nn, (void*)&H, &lh, &wk, &D, &Y, &ly, (void*)&ri};
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
