// Step 9 of Algorithm 2 (H Y = Y D, float64) by the tridiagonal route, for 32 < n <= kTrdMaxN.
//
// GB300 retires two float64 FMA per clock per SM, so the flop count matters more than on
// earlier parts: cyclic Jacobi spends some 30 n^3 flops (about ten sweeps), while this route
// spends about 4 n^3, most of it on the whole GPU.
//
//  1. trd_reduce_kernel, one thread-block cluster of kTrdCl CTAs.  H sits in the CTAs'
//     shared memory, row r in CTA r mod kTrdCl.  Householder reflections P_i = I - tau_i v_i
//     v_i^T reduce it to tridiagonal T = Q^T H Q (A <- A - v w^T - w v^T with
//     p = tau A v, w = p - (tau/2)(p^T v) v).  Each column costs two cluster barriers: the
//     owners push the next column (and partial sums of its squares) and the entries of p (and
//     partial p^T v) into every CTA's shared memory before the barrier, so nothing is fetched
//     after one.  Q = P_0 P_1 ... P_{n-3} is then accumulated backwards with Q held by columns
//     (column c in CTA c mod kTrdCl): w^T = v^T Q and Q <- Q - tau v w^T need no exchange, only
//     v, read from the owners of the rows.  T splits where |e_i| <= eps ||T||.
//  2. trd_bisect_kernel, one warp per eigenvalue: multisection (64 points per round) on Sturm
//     counts (signs of the leading minors of T - x I) of the eigenvalue's block of T.
//  3. trd_vectors_kernel, one warp per eigenvalue: inverse iteration (two solves with T - lambda
//     I, LU with partial pivoting) from a pseudo-random start.  Eigenvalues closer than
//     kTrdTightGap ||T|| to a neighbour form a tight cluster: its leader iterates on all of its
//     columns at once and orthonormalises them within the cluster after each solve (the
//     cluster's invariant subspace, in which any orthonormal basis is an eigenbasis to within
//     the cluster's width).  Independent solves leave the eigenvectors of close but separated
//     eigenvalues non-orthogonal by about eps ||T|| / gap.
//  4. trd_gemm_kernel: G = Z^T Z and P = Q Z in one launch, then Y = P (3 I - G) / 2 (one
//     Newton-Schulz step towards the orthogonal polar factor, quadratic in Z^T Z - I), the
//     columns written in ascending order of the eigenvalues.
//
// The route reports, for the parallel Jacobi kernel that follows it, whether its result is to
// be replaced: a non-finite H, a tight cluster wider than kTrdMaxWidth ||T||, or Z^T Z - I
// larger than kTrdMaxOrth (where one Newton-Schulz step is not enough).
#include <cooperative_groups.h>

#include <algorithm>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace bchdav {

namespace {

constexpr int kTrdCl = 16;          // CTAs per cluster (non-portable size, checked at set-up)
constexpr int kTrdThreads = 256;
constexpr int kTrdMaxRows = (kTrdMaxN + kTrdCl - 1) / kTrdCl;
constexpr double kTrdEps = 2.220446049250313e-16;
constexpr double kTrdTightGap = 1e-10;   // relative to ||T||
constexpr double kTrdMaxWidth = 1e3 * kTrdEps;
constexpr double kTrdMaxOrth = 1e-7;

// control words at the end of the work area
struct TrdCtl {
  double tnorm;
  unsigned long long g0;   // bits of max |Z^T Z - I| (non-negative doubles order as integers)
  int fallback;            // set by the route's kernels when its result is to be replaced
  int run_jacobi;          // decision for the kernel that follows (written last)
};

struct TrdLayout {
  double *Q, *Zt, *P, *G, *Vr, *tau, *d, *e, *dn, *e2n, *lam, *scr;
  int *bstart, *bend, *rank;
  TrdCtl* ctl;
};

__host__ __device__ inline TrdLayout trd_layout(double* w, int n) {
  TrdLayout L;
  const size_t nn = (size_t)n * n;
  L.Q = w;
  L.Zt = L.Q + nn;
  L.P = L.Zt + nn;
  L.G = L.P + nn;
  L.Vr = L.G + nn;              // reflector i in row i (entries i+1 .. n-1)
  L.tau = L.Vr + nn;
  L.scr = L.tau + n;            // 6 n per eigenvalue: LU factors of T - lambda I
  L.d = L.scr + 6 * nn;
  L.e = L.d + n;
  L.dn = L.e + n;               // d / ||T||
  L.e2n = L.dn + n;             // (e / ||T||)^2
  L.lam = L.e2n + n;
  L.bstart = reinterpret_cast<int*>(L.lam + n);
  L.bend = L.bstart + n;
  L.rank = L.bend + n;
  L.ctl = reinterpret_cast<TrdCtl*>(L.lam + n + (3 * (size_t)n + 1) / 2 + 2);
  return L;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double trd_block_sum(double v, double* s_red) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kTrdThreads / 32; ++w) s += s_red[w];
  __syncthreads();   // s_red is reused
  return s;
}

// shared-memory layout of trd_reduce_kernel (doubles)
struct TrdSmem {
  double* A;      // own rows of the working matrix, kTrdMaxRows x ldA
  double* xb;     // [2][n] the column being reduced (pushed by its owners), by parity
  double* pf;     // [n] p = tau A v, pushed by its owners
  double* w;      // [n] w = p - K v
  double* taus;   // [n]
  double* sq;     // [kTrdCl] partial sums of squares of the pushed column
  double* pv;     // [kTrdCl] partial p^T v
  double* red;    // [64]
  double* rowv;   // [32] one value per own row (p_r v_r, or a squared entry)
  double* sraw;   // [32] A x for own rows, x the column before scaling
  double* sc;     // [8] scalars of the current column: tau, scale, beta, K, 1 - scale alpha
};

__host__ __device__ inline size_t trd_smem_doubles(int n) {
  const int ldA = n | 1;
  return (size_t)kTrdMaxRows * ldA + 5 * (size_t)n + 2 * (size_t)kTrdCl + 64 + 32 + 32 + 8;
}

__device__ inline TrdSmem trd_smem(double* base, int n) {
  TrdSmem S;
  const int ldA = n | 1;
  S.A = base;
  S.xb = S.A + (size_t)kTrdMaxRows * ldA;
  S.pf = S.xb + 2 * n;
  S.w = S.pf + n;
  S.taus = S.w + n;
  S.sq = S.taus + n;
  S.pv = S.sq + kTrdCl;
  S.red = S.pv + kTrdCl;
  S.rowv = S.red + 64;
  S.sraw = S.rowv + 32;
  S.sc = S.sraw + 32;
  return S;
}

// Writes `val` to offset `off` of every CTA's copy of the array `local` (the same shared-memory
// offset in each CTA of the cluster).
__device__ __forceinline__ void trd_push(cg::cluster_group& cl, double* local, int off, double val) {
#pragma unroll 4
  for (int c = 0; c < kTrdCl; ++c) cl.map_shared_rank(local, c)[off] = val;
}

// Dot products of R rows (or columns) of a warp with one vector, two accumulators per row,
// reduced together across the lanes: R independent dependent chains instead of one.
template <int R>
__device__ __forceinline__ void trd_dots(const double* const (&row)[4], const double* __restrict__ x,
                                         int m, int lane, double (&out)[4]) {
  double acc[R][2];
#pragma unroll
  for (int u = 0; u < R; ++u) acc[u][0] = acc[u][1] = 0.0;
  for (int q = lane; q < m; q += 64) {
    const double x0 = x[q];
    const bool two = q + 32 < m;
    const double x1 = two ? x[q + 32] : 0.0;
    const int q1 = two ? q + 32 : q;
#pragma unroll
    for (int u = 0; u < R; ++u) {
      acc[u][0] = fma(row[u][q], x0, acc[u][0]);
      acc[u][1] = fma(row[u][q1], x1, acc[u][1]);
    }
  }
#pragma unroll
  for (int u = 0; u < R; ++u) out[u] = acc[u][0] + acc[u][1];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int u = 0; u < R; ++u) out[u] += __shfl_xor_sync(0xffffffffu, out[u], o);
  }
}

__device__ __forceinline__ void trd_dots_n(int cnt, const double* const (&row)[4],
                                           const double* __restrict__ x, int m, int lane,
                                           double (&out)[4]) {
  switch (cnt) {   // warp-uniform
    case 4: trd_dots<4>(row, x, m, lane, out); break;
    case 3: trd_dots<3>(row, x, m, lane, out); break;
    case 2: trd_dots<2>(row, x, m, lane, out); break;
    case 1: trd_dots<1>(row, x, m, lane, out); break;
    default: break;
  }
}

__global__ void __launch_bounds__(kTrdThreads, 1)
    trd_reduce_kernel(int n, const double* __restrict__ H, int ldh, TrdLayout L) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double sm_trd[];
  TrdSmem S = trd_smem(sm_trd, n);
  const int me = (int)cl.block_rank();
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int ldA = n | 1;
  const int nown = (n - me + kTrdCl - 1) / kTrdCl;   // own rows r = me + kTrdCl * lr
  cl.sync();   // every CTA of the cluster runs before any shared memory is written remotely
  // own rows of H (upper triangle read, mirrored), own columns of Q = I
  for (int idx = t; idx < nown * n; idx += kTrdThreads) {
    const int lr = idx / n, c = idx - lr * n, r = me + kTrdCl * lr;
    S.A[lr * ldA + c] = (r <= c) ? H[(size_t)r * ldh + c] : H[(size_t)c * ldh + r];
  }
  // column 0 (rows 1..n-1) goes to every CTA's xb[0] by its owners, with partial squares of
  // rows 2..n-1
  __syncthreads();
  {
    double sq = 0.0;
    for (int lr = t; lr < nown; lr += kTrdThreads) {
      const int r = me + kTrdCl * lr;
      if (r >= 1) {
        const double x = S.A[lr * ldA + 0];
        trd_push(cl, S.xb, r - 1, x);
        if (r >= 2) sq = fma(x, x, sq);
      }
    }
    sq = trd_block_sum(sq, S.red);
    if (t == 0) trd_push(cl, S.sq, me, sq);
  }
  cl.sync();
  double tn = 0.0;   // running max of |d_i| + |e_{i-1}| + |e_i| (CTA 0, thread 32)
  double e_prev = 0.0;
  // GB300's float64 pipe is narrow and its results come late, so a column's critical path is a
  // count of dependent float64 operations.  Scalar work (square root, divisions, sums over the
  // CTAs or the own rows) is done by one warp and handed to the others through shared memory;
  // the matrix-vector product starts from the unscaled column x at once, beside that warp:
  // A v = scale A x + (1 - scale alpha) A e_0, as v = scale x except v_0 = 1.  Dot products keep
  // two accumulators per row and a warp's rows (at most four) are reduced together.
  constexpr int kRowsW = (kTrdMaxRows + 6) / 7;   // own rows per warp 1..7
  for (int i = 0; i < n - 2; ++i) {
    const int m = n - i - 1;   // trailing size: rows / columns i+1 .. n-1
    double* x = S.xb + (i & 1) * n;
    const int lr0 = (i + 1 - me + kTrdCl - 1) / kTrdCl;   // first own row > i
    if (warp == 0) {
      // reflector from the pushed column x = A(i+1:n-1, i)
      const double sig = warp_sum(lane < kTrdCl ? S.sq[lane] : 0.0);
      if (lane == 0) {
        const double alpha = x[0];
        double tau = 0.0, beta = alpha, scale = 0.0;
        if (sig != 0.0) {
          beta = -copysign(sqrt(fma(alpha, alpha, sig)), alpha);
          tau = (beta - alpha) / beta;
          scale = 1.0 / (alpha - beta);
        }
        S.sc[0] = tau;
        S.sc[1] = scale;
        S.sc[2] = beta;
        S.sc[4] = (sig != 0.0) ? fma(-scale, alpha, 1.0) : 1.0;
        S.taus[i] = tau;
      }
    } else {
      // raw products A(r, i+1:n-1) x for the own rows lr0 + (warp - 1) + 7 u
      const int first = lr0 + warp - 1;
      const int cnt = first < nown ? min(kRowsW, (nown - first + 6) / 7) : 0;
      const double* Ar[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) Ar[u] = S.A + (u < cnt ? first + 7 * u : 0) * ldA + i + 1;
      double sum[4];
      trd_dots_n(cnt, Ar, x, m, lane, sum);
      if (lane == 0)
        for (int u = 0; u < cnt; ++u) S.sraw[first + 7 * u] = sum[u];
    }
    __syncthreads();
    const double tau = S.sc[0], scale = S.sc[1], c0 = S.sc[4];
    // p = tau A v on own rows (one thread per row and destination CTA); v into column i
    for (int idx = t; idx < (nown - lr0) * kTrdCl; idx += kTrdThreads) {
      const int lr = lr0 + idx / kTrdCl, dst = idx % kTrdCl;
      const int r = me + kTrdCl * lr, qr = r - i - 1;
      const double p = tau * fma(scale, S.sraw[lr], c0 * S.A[lr * ldA + i + 1]);
      cl.map_shared_rank(S.pf, dst)[qr] = p;
      if (dst == 0) {
        const double vr = (qr == 0) ? 1.0 : x[qr] * scale;
        S.A[lr * ldA + i] = vr;
        S.rowv[lr] = p * vr;
      }
    }
    if (me == 0 && t == 32) {
      const double di = cl.map_shared_rank(S.A, i % kTrdCl)[(i / kTrdCl) * ldA + i];
      const double beta = S.sc[2];
      L.d[i] = di;
      L.e[i] = beta;
      tn = fmax(tn, fabs(di) + fabs(e_prev) + fabs(beta));
      e_prev = beta;
    }
    __syncthreads();   // A(:, i) holds v before x is scaled in place
    for (int q = t; q < m; q += kTrdThreads) x[q] = (q == 0) ? 1.0 : x[q] * scale;
    if (warp == 0) {
      const double pvp = warp_sum((lr0 + lane < nown) ? S.rowv[lr0 + lane] : 0.0);
      if (lane < kTrdCl) cl.map_shared_rank(S.pv, lane)[me] = pvp;
    }
    cl.sync();
    // w = p - (tau / 2) (p^T v) v
    if (warp == 0) {
      const double ptv = warp_sum(lane < kTrdCl ? S.pv[lane] : 0.0);
      if (lane == 0) S.sc[3] = 0.5 * tau * ptv;
    }
    __syncthreads();
    {
      const double K = S.sc[3];
      for (int q = t; q < m; q += kTrdThreads) S.w[q] = fma(-K, x[q], S.pf[q]);
    }
    __syncthreads();
    // A <- A - v w^T - w v^T on own rows > i; column i + 1 first, pushed with its squares
    double* xn = S.xb + ((i + 1) & 1) * n;
    for (int lr = lr0 + t; lr < nown; lr += kTrdThreads) {
      const int r = me + kTrdCl * lr, qr = r - i - 1;
      double* a = S.A + lr * ldA + i + 1;   // entry (r, i + 1)
      const double val = a[0] - x[qr] * S.w[0] - S.w[qr] * x[0];
      a[0] = val;
      if (r >= i + 2) trd_push(cl, xn, r - i - 2, val);
      S.rowv[lr] = (r >= i + 3) ? val * val : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      const double sqn = warp_sum((lr0 + lane < nown) ? S.rowv[lr0 + lane] : 0.0);
      if (lane < kTrdCl) cl.map_shared_rank(S.sq, lane)[me] = sqn;
    }
    for (int lr = lr0 + warp; lr < nown; lr += kTrdThreads / 32) {
      const int r = me + kTrdCl * lr, qr = r - i - 1;
      const double vr = x[qr], wr = S.w[qr];
      double* a = S.A + lr * ldA + i + 1;
#pragma unroll 4
      for (int q = 1 + lane; q < m; q += 32) a[q] = fma(-wr, x[q], fma(-vr, S.w[q], a[q]));
    }
    cl.sync();
  }
  // the last 2 x 2 block
  if (me == 0 && t == 32) {
    const double a22 = cl.map_shared_rank(S.A, (n - 2) % kTrdCl)[((n - 2) / kTrdCl) * ldA + n - 2];
    const double a33 = cl.map_shared_rank(S.A, (n - 1) % kTrdCl)[((n - 1) / kTrdCl) * ldA + n - 1];
    const double a32 = cl.map_shared_rank(S.A, (n - 1) % kTrdCl)[((n - 1) / kTrdCl) * ldA + n - 2];
    L.d[n - 2] = a22;
    L.d[n - 1] = a33;
    L.e[n - 2] = a32;
    L.e[n - 1] = 0.0;
    tn = fmax(tn, fabs(a22) + fabs(e_prev) + fabs(a32));
    tn = fmax(tn, fabs(a33) + fabs(a32));
    S.sc[4] = tn;
  }
  __syncthreads();
  if (me == 0) {
    // splits (|e_k| <= eps ||T||) and the scaled copies, then the blocks
    const double tn = S.sc[4];
    const double itn = 1.0 / tn;
    const double thr = kTrdEps * tn;
    for (int k = t; k < n; k += kTrdThreads) {
      double ek = L.e[k];
      if (k == n - 1 || fabs(ek) <= thr) ek = 0.0;
      L.e[k] = ek;
      const double en = ek * itn;
      L.e2n[k] = en * en;
      L.dn[k] = L.d[k] * itn;
    }
    __syncthreads();
    if (t == 0) {
      int s0 = 0;
      for (int k = 0; k < n; ++k) {
        if (k == n - 1 || L.e[k] == 0.0) {
          for (int u = s0; u <= k; ++u) {
            L.bstart[u] = s0;
            L.bend[u] = k + 1;
          }
          s0 = k + 1;
        }
      }
      L.ctl->tnorm = tn;
      L.ctl->fallback = !(tn < INFINITY);   // also catches NaN
      L.ctl->g0 = 0ull;
      L.ctl->run_jacobi = 0;
    }
  }
  // the reflectors for trd_qform_kernel: v_i (rows i+1 .. n-1, v_i(i+1) = 1) into row i of Vr
  for (int idx = t; idx < nown * n; idx += kTrdThreads) {
    const int lr = idx / n, i = idx - lr * n, r = me + kTrdCl * lr;
    if (i < r - 1) L.Vr[(size_t)i * n + r] = S.A[lr * ldA + i];
    else if (i == r - 1) L.Vr[(size_t)i * n + r] = 1.0;
  }
  if (me == 0)
    for (int i = t; i < n; i += kTrdThreads) L.tau[i] = (i < n - 2) ? S.taus[i] : 0.0;
  cl.sync();   // no CTA leaves while others may still read its shared memory
}

// Q = P_0 P_1 ... P_{n-3}, accumulated backwards (Q <- P_i Q touches rows and columns i+1 ..
// n-1), columns distributed over the CTAs (column c in CTA c mod gridDim.x, held in shared
// memory): w^T = v^T Q and Q <- Q - tau v w^T need no exchange, only v_i, read from the
// reflector rows that trd_reduce_kernel wrote (the next one fetched while the current one is
// applied).  It runs beside the eigenvalue and eigenvector kernels, on another stream.
constexpr int kQfCtas = 32;

__global__ void __launch_bounds__(kTrdThreads) trd_qform_kernel(int n, TrdLayout L) {
  extern __shared__ double sm_qf[];
  const int me = blockIdx.x, G = gridDim.x;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int ncol = (n - me + G - 1) / G;        // own columns c = me + G lc
  double* Qc = sm_qf;                           // ncol x n, column-major
  double* vq = Qc + (size_t)((n + G - 1) / G) * n;   // [2][n]
  for (int idx = t; idx < ncol * n; idx += kTrdThreads) {
    const int lc = idx / n, r = idx - lc * n;
    Qc[lc * n + r] = (r == me + G * lc) ? 1.0 : 0.0;
  }
  auto fetch_v = [&](int i, double* dst) {
    const int m = n - i - 1;
    for (int q = t; q < m; q += kTrdThreads) dst[q] = __ldcg(L.Vr + (size_t)i * n + i + 1 + q);
  };
  if (n >= 3) fetch_v(n - 3, vq + ((n - 3) & 1) * n);
  for (int i = n - 3; i >= 0; --i) {
    __syncthreads();   // v_i complete; the other buffer is free
    if (i >= 1) fetch_v(i - 1, vq + ((i - 1) & 1) * n);
    const double tau = __ldcg(L.tau + i);
    if (tau == 0.0) continue;
    const double* v = vq + (i & 1) * n;
    const int m = n - i - 1;
    const int lc0 = (i + 1 - me + G - 1) / G;   // first own column > i
    const int first = lc0 + warp;
    const int cnt = first < ncol ? min(4, (ncol - first + 7) / 8) : 0;
    const double* qr[4];
    double* qc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      qc[u] = Qc + (u < cnt ? first + 8 * u : 0) * n + i + 1;   // rows i+1 .. n-1
      qr[u] = qc[u];
    }
    double f[4];
    trd_dots_n(cnt, qr, v, m, lane, f);
    for (int u = 0; u < cnt; ++u) {
      const double fu = tau * f[u];
#pragma unroll 4
      for (int q = lane; q < m; q += 32) qc[u][q] = fma(-fu, v[q], qc[u][q]);
    }
  }
  __syncthreads();
  for (int idx = t; idx < ncol * n; idx += kTrdThreads) {
    const int lc = idx / n, r = idx - lc * n;
    L.Q[(size_t)r * n + me + G * lc] = Qc[lc * n + r];
  }
}

// Number of eigenvalues of the block [s0, s1) of T / ||T|| below x0 and below x1: the sign
// changes of the leading principal minors P_0 = 1, P_i = (d_i - x) P_{i-1} - e_{i-1}^2 P_{i-2}
// (the Sturm sequence).  A P_i that is exactly zero takes the sign opposite to P_{i-1} (as a
// pivot of the LDL^T factorisation of T - x I that is taken negative), magnitude |P_{i-1}|
// 2^-600, set with integer operations so that the dependent chain from one minor to the next
// is a single float64 FMA; the two shifts' chains are interleaved.  |P_i / P_{i-1}| <= 3 on
// the scaled matrix, so a rescaling by a power of two every eight entries keeps them in range.
__device__ __forceinline__ double trd_nonzero(double pn, double pc) {
  const int hi = __double2hiint(pn), lo = __double2loint(pn);
  const int hp = __double2hiint(pc);
  const int ex = (hp >> 20) & 0x7ff;
  const double alt = __hiloint2double((~hp & (int)0x80000000) | ((ex > 601 ? ex - 600 : 1) << 20), 0);
  return (((hi & 0x7fffffff) | lo) == 0) ? alt : pn;
}

__device__ __forceinline__ void trd_rescale(double& pc, double& pm) {
  const int ex = ((__double2hiint(pc) >> 20) & 0x7ff) - 1023;
  if (ex > 300 || ex < -300) {
    const double f = __hiloint2double((1023 - ex) << 20, 0);   // 2^-ex
    pc *= f;
    pm *= f;
  }
}

__device__ __forceinline__ void trd_sturm2(const double* __restrict__ dn,
                                           const double* __restrict__ e2n, int s0, int s1,
                                           double x0, double x1, int& c0, int& c1) {
  double pm0 = 1.0, pm1 = 1.0;
  double pc0 = trd_nonzero(dn[s0] - x0, pm0), pc1 = trd_nonzero(dn[s0] - x1, pm1);
  c0 = pc0 < 0.0;
  c1 = pc1 < 0.0;
  for (int i = s0 + 1; i < s1; ++i) {
    const double di = dn[i], ei = e2n[i - 1];
    double pn0 = fma(di - x0, pc0, -ei * pm0);
    double pn1 = fma(di - x1, pc1, -ei * pm1);
    pn0 = trd_nonzero(pn0, pc0);
    pn1 = trd_nonzero(pn1, pc1);
    c0 += (__double2hiint(pn0) ^ __double2hiint(pc0)) < 0;
    c1 += (__double2hiint(pn1) ^ __double2hiint(pc1)) < 0;
    pm0 = pc0;
    pc0 = pn0;
    pm1 = pc1;
    pc1 = pn1;
    if (((i - s0) & 7) == 0) {
      trd_rescale(pc0, pm0);
      trd_rescale(pc1, pm1);
    }
  }
}

// one warp per eigenvalue in the vector kernel, two warps per CTA (the float64 pipes of all SMs)
constexpr int kTrdEigWarps = 2;

// Multisection, one warp per eigenvalue (one warp per CTA): each lane counts at two points, so
// a round places 64 points in the interval (6 bits per round, 9 rounds for float64).  The
// rounds are bound by the latency of the Sturm chain, not by float64 throughput.
__global__ void __launch_bounds__(32) trd_bisect_kernel(int n, TrdLayout L) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x;
  if (j >= n) return;
  const int s0 = L.bstart[j], s1 = L.bend[j], k = j - s0;
  if (s1 - s0 == 1) {
    if (lane == 0) L.lam[j] = L.d[s0];
    return;
  }
  const double tn = L.ctl->tnorm;
  const double* dn = L.dn;
  const double* e2n = L.e2n;
  // Gershgorin interval of the block, on the scaled matrix
  double lo = INFINITY, hi = -INFINITY;
  for (int i = s0 + lane; i < s1; i += 32) {
    const double el = (i > s0) ? sqrt(e2n[i - 1]) : 0.0;
    const double er = (i < s1 - 1) ? sqrt(e2n[i]) : 0.0;
    lo = fmin(lo, dn[i] - el - er);
    hi = fmax(hi, dn[i] + el + er);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  lo -= 4.0 * kTrdEps;
  hi += 4.0 * kTrdEps;
  const double atol = 0.5 * kTrdEps;   // of ||T||
  for (int round = 0; round < 64; ++round) {
    const double width = hi - lo;
    if (!(width > fmax(2.0 * kTrdEps * fmax(fabs(lo), fabs(hi)), atol))) break;
    // points p = 2 lane + c, c = 0, 1, at lo + width (p + 1) / 65
    const double x0 = lo + width * ((double)(2 * lane + 1) * (1.0 / 65.0));
    const double x1 = lo + width * ((double)(2 * lane + 2) * (1.0 / 65.0));
    int c0, c1;
    trd_sturm2(dn, e2n, s0, s1, x0, x1, c0, c1);
    const unsigned a0 = __ballot_sync(0xffffffffu, c0 > k), a1 = __ballot_sync(0xffffffffu, c1 > k);
    // first point whose count exceeds k: the eigenvalue lies below it, above the one before
    const int f0 = a0 ? 2 * (__ffs(a0) - 1) : 64, f1 = a1 ? 2 * (__ffs(a1) - 1) + 1 : 64;
    const int first = min(f0, f1);
    const double xf0 = __shfl_sync(0xffffffffu, x0, (first >> 1) & 31);
    const double xf1 = __shfl_sync(0xffffffffu, x1, (first >> 1) & 31);
    const int prev = first - 1;
    const double xp0 = __shfl_sync(0xffffffffu, x0, (prev >> 1) & 31);
    const double xp1 = __shfl_sync(0xffffffffu, x1, (prev >> 1) & 31);
    const double nhi = (first == 64) ? hi : ((first & 1) ? xf1 : xf0);
    const double nlo = (first == 0) ? lo : ((prev & 1) ? xp1 : xp0);
    if (!(nhi - nlo < width)) break;   // no progress (rounding)
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) L.lam[j] = 0.5 * (lo + hi) * tn;
}

// LU factors with partial pivoting of T_b - lambda I (block [s0, s1)): the elimination of a
// tridiagonal matrix with row interchanges fills one extra superdiagonal.  f holds 6 nb doubles:
// reciprocal pivots, the two superdiagonals of U, the multipliers and the interchanges.
__device__ void trd_factor(const double* __restrict__ d, const double* __restrict__ e, int s0,
                           int s1, double lambda, double tiny, double* __restrict__ f) {
  const int nb = s1 - s0;
  double* rp = f;             // 1 / pivot
  double* du = f + nb;        // first superdiagonal of U
  double* du2 = f + 2 * nb;   // second superdiagonal of U
  double* mul = f + 3 * nb;   // multipliers
  double* swp = f + 4 * nb;   // 1: rows i and i + 1 were interchanged
  double dcur = d[s0] - lambda;   // pivot candidate of row i
  double ucur = (nb > 1) ? e[s0] : 0.0;
  for (int i = 0; i < nb - 1; ++i) {
    const double sub = e[s0 + i];   // entry (i + 1, i)
    const double dnext = d[s0 + i + 1] - lambda;
    const double unext = (i < nb - 2) ? e[s0 + i + 1] : 0.0;
    if (fabs(dcur) >= fabs(sub)) {
      const double piv = (dcur == 0.0) ? tiny : dcur;
      const double m = sub / piv;
      rp[i] = 1.0 / piv;
      du[i] = ucur;
      du2[i] = 0.0;
      mul[i] = m;
      swp[i] = 0.0;
      dcur = dnext - m * ucur;
      ucur = unext;
    } else {
      const double m = dcur / sub;
      rp[i] = 1.0 / sub;
      du[i] = dnext;
      du2[i] = unext;
      mul[i] = m;
      swp[i] = 1.0;
      dcur = ucur - m * dnext;
      ucur = -m * unext;
    }
  }
  rp[nb - 1] = 1.0 / ((dcur == 0.0) ? tiny : dcur);
  du[nb - 1] = 0.0;
  du2[nb - 1] = 0.0;
}

// y <- (T_b - lambda I)^{-1} y from the factors of trd_factor
__device__ void trd_lu_solve(int nb, const double* __restrict__ f, double* __restrict__ y) {
  const double* rp = f;
  const double* du = f + nb;
  const double* du2 = f + 2 * nb;
  const double* mul = f + 3 * nb;
  const double* swp = f + 4 * nb;
  for (int i = 0; i < nb - 1; ++i) {
    if (swp[i] != 0.0) {
      const double yi = y[i];
      y[i] = y[i + 1];
      y[i + 1] = fma(-mul[i], y[i + 1], yi);
    } else {
      y[i + 1] = fma(-mul[i], y[i], y[i + 1]);
    }
  }
  y[nb - 1] *= rp[nb - 1];
  if (nb > 1) y[nb - 2] = (y[nb - 2] - du[nb - 2] * y[nb - 1]) * rp[nb - 2];
  for (int i = nb - 3; i >= 0; --i) y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) * rp[i];
}

// pseudo-random start entry in [-1, 1) of eigenvector slot j, row i (Philox4x32-10)
__device__ __forceinline__ double trd_start(int j, int i) {
  U4 c = {(uint32_t)i, (uint32_t)j, 0x7e1dU, 0u};
  U4 r = philox4x32_10(c, 0x2212u, 0x04443u);
  const uint64_t u = ((uint64_t)r.x << 21) ^ (uint64_t)r.y;   // 53 random bits
  return (double)(u & ((1ull << 53) - 1)) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void __launch_bounds__(kTrdEigWarps * 32) trd_vectors_kernel(int n, TrdLayout L) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * kTrdEigWarps + (threadIdx.x >> 5);
  if (j >= n) return;
  const int s0 = L.bstart[j], s1 = L.bend[j], nb = s1 - s0, k = j - s0;
  const double tn = L.ctl->tnorm;
  const double* lam = L.lam;
  // rank of each eigenvalue among all: ascending, ties by slot
  auto rank_of = [&](int jj) {
    const double lj = lam[jj];
    int rk = 0;
    for (int i = lane; i < n; i += 32) rk += (lam[i] < lj) || (lam[i] == lj && i < jj);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rk += __shfl_xor_sync(0xffffffffu, rk, o);
    return rk;
  };
  // tight cluster: chains of gaps <= kTrdTightGap ||T|| inside the block; its first member leads
  const double gap = kTrdTightGap * tn;
  if (k > 0 && !(lam[j] - lam[j - 1] > gap)) return;
  int c = 1;
  while (k + c < nb && !(lam[j + c] - lam[j + c - 1] > gap)) ++c;
  for (int q = 0; q < c; ++q) {
    const int rk = rank_of(j + q);
    if (lane == 0) L.rank[j + q] = rk;
  }
  if (c > 1 && lam[j + c - 1] - lam[j] > kTrdMaxWidth * tn && lane == 0)
    atomicOr(&L.ctl->fallback, 1);
  // rows outside the block are zero
  for (int q = 0; q < c; ++q) {
    double* z = L.Zt + (size_t)(j + q) * n;
    for (int i = lane; i < n; i += 32)
      if (i < s0 || i >= s1) z[i] = 0.0;
  }
  const double tiny = kTrdEps * tn + 1e-300;
  if (nb == 1) {
    if (lane == 0) L.Zt[(size_t)j * n + s0] = 1.0;
    return;
  }
  // start vectors, then two rounds of (solve, orthonormalise within the cluster)
  for (int q = 0; q < c; ++q) {
    double* z = L.Zt + (size_t)(j + q) * n + s0;
    for (int i = lane; i < nb; i += 32) z[i] = trd_start(j + q, i);
  }
  for (int q = lane; q < c; q += 32)
    trd_factor(L.d, L.e, s0, s1, lam[j + q], tiny, L.scr + (size_t)(j + q) * 6 * n);
  __syncwarp();
  for (int it = 0; it < 2; ++it) {
    for (int q = lane; q < c; q += 32)
      trd_lu_solve(nb, L.scr + (size_t)(j + q) * 6 * n, L.Zt + (size_t)(j + q) * n + s0);
    __syncwarp();
    // Gram-Schmidt inside the cluster, twice; normalisation
    for (int rep = 0; rep < (c > 1 ? 2 : 1); ++rep) {
      for (int q = 0; q < c; ++q) {
        double* zq = L.Zt + (size_t)(j + q) * n + s0;
        for (int p = 0; p < q; ++p) {
          const double* zp = L.Zt + (size_t)(j + p) * n + s0;
          double s = 0.0;
          for (int i = lane; i < nb; i += 32) s = fma(zp[i], zq[i], s);
          s = warp_sum(s);
          for (int i = lane; i < nb; i += 32) zq[i] = fma(-s, zp[i], zq[i]);
          __syncwarp();
        }
        double s = 0.0;
        for (int i = lane; i < nb; i += 32) s = fma(zq[i], zq[i], s);
        s = warp_sum(s);
        const double inv = 1.0 / sqrt(s);
        if (!(inv < INFINITY) || !(s > 0.0)) {
          if (lane == 0) atomicOr(&L.ctl->fallback, 1);
        }
        for (int i = lane; i < nb; i += 32) zq[i] *= inv;
        __syncwarp();
      }
    }
  }
}

// C = A B^T over n x n row-major operands (ld n), 16 x 16 output tiles, k in chunks of 32.
// MODE 0: blockIdx.z = 0: G = Zt Zt^T (and max |G - I|), 1: P = Q Zt^T.
// MODE 1: Y(:, rank(j)) = 1.5 P(:, j) - 0.5 (P G^T)(:, j), D(rank(j)) = lambda_j.
template <int MODE>
__global__ void __launch_bounds__(256) trd_gemm_kernel(int n, TrdLayout L, double* __restrict__ D,
                                                       double* __restrict__ Y, int ldy) {
  __shared__ double As[16][33];
  __shared__ double Bs[16][33];
  __shared__ double s_max[8];
  const double* A;
  const double* B;
  if (MODE == 0) {
    A = blockIdx.z == 0 ? L.Zt : L.Q;
    B = L.Zt;
  } else {
    A = L.P;
    B = L.G;
  }
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int idx = t; idx < 16 * 32; idx += 256) {
      const int r = idx >> 5, kk = idx & 31, k = k0 + kk;
      As[r][kk] = (i0 + r < n && k < n) ? A[(size_t)(i0 + r) * n + k] : 0.0;
      Bs[r][kk] = (j0 + r < n && k < n) ? B[(size_t)(j0 + r) * n + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) acc = fma(As[ty][kk], Bs[tx][kk], acc);
    __syncthreads();
  }
  const int i = i0 + ty, j = j0 + tx;
  const bool in = i < n && j < n;
  if (MODE == 0) {
    if (blockIdx.z == 0) {
      if (in) L.G[(size_t)i * n + j] = acc;
      double dev = in ? fabs(acc - (i == j ? 1.0 : 0.0)) : 0.0;
      if (!(dev == dev)) dev = INFINITY;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
      if ((t & 31) == 0) s_max[t >> 5] = dev;
      __syncthreads();
      if (t == 0) {
        double mx = 0.0;
        for (int w = 0; w < 8; ++w) mx = fmax(mx, s_max[w]);
        atomicMax(&L.ctl->g0, (unsigned long long)__double_as_longlong(mx));
      }
    } else if (in) {
      L.P[(size_t)i * n + j] = acc;
    }
  } else {
    if (in) {
      const int rk = L.rank[j];
      Y[(size_t)i * ldy + rk] = fma(1.5, L.P[(size_t)i * n + j], -0.5 * acc);
      if (i == 0) D[rk] = L.lam[j];
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && t == 0) {
      const double g0 = __longlong_as_double((long long)L.ctl->g0);
      L.ctl->run_jacobi = (L.ctl->fallback != 0 || !(g0 <= kTrdMaxOrth)) ? 1 : 0;
    }
  }
}

}  // namespace

size_t trd_work_doubles(int n) {
  const size_t nn = (size_t)n * n;
  return 11 * nn + 6 * (size_t)n + (3 * (size_t)n + 1) / 2 + 2 + sizeof(TrdCtl) / sizeof(double) + 4;
}

// 0 when this device cannot co-schedule the cluster (the caller keeps the Jacobi route)
static int trd_cluster_ok(int n) {
  // decided once, at the first call (for the largest shared memory, n = kTrdMaxN)
  static const int ok = []() {
    const size_t smem = trd_smem_doubles(kTrdMaxN) * sizeof(double);
    int v = 0;
    if (cudaFuncSetAttribute(trd_reduce_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess &&
        cudaFuncSetAttribute(trd_reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(kTrdCl, 1, 1);
      cfg.blockDim = dim3(kTrdThreads, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = kTrdCl;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, trd_reduce_kernel, &cfg) == cudaSuccess &&
          clusters >= 1)
        v = 1;
    }
    cudaGetLastError();
    return v;
  }();
  return (n > 32 && n <= kTrdMaxN) ? ok : 0;
}

cudaError_t launch_trd_eigh(cudaStream_t st, int n, const double* H, int ldh, double* D,
                            double* Y, int ldy, double* work, int** run_jacobi, cudaStream_t aux,
                            cudaEvent_t ev_reduced, cudaEvent_t ev_q) {
  *run_jacobi = nullptr;
  if (!trd_cluster_ok(n)) return cudaErrorNotSupported;
  TrdLayout L = trd_layout(work, n);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kTrdCl, 1, 1);
  cfg.blockDim = dim3(kTrdThreads, 1, 1);
  cfg.dynamicSmemBytes = trd_smem_doubles(n) * sizeof(double);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kTrdCl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  note_launch();
  cudaError_t e = cudaLaunchKernelEx(&cfg, trd_reduce_kernel, n, H, ldh, L);
  if (e != cudaSuccess) return e;
  // Q's accumulation beside the eigenvalues and vectors of T (another stream when given)
  const size_t qf_smem = ((size_t)ceil_div(n, kQfCtas) * n + 2 * (size_t)n) * sizeof(double);
  static const bool qf_attr = [] {
    return cudaFuncSetAttribute(trd_qform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(((size_t)ceil_div(kTrdMaxN, kQfCtas) * kTrdMaxN +
                                       2 * (size_t)kTrdMaxN) * sizeof(double))) == cudaSuccess;
  }();
  if (!qf_attr) return cudaErrorInvalidValue;
  const bool fork = aux != nullptr && ev_reduced != nullptr && ev_q != nullptr;
  cudaStream_t sq = fork ? aux : st;
  if (fork) {
    e = cudaEventRecord(ev_reduced, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev_reduced, 0);
    if (e != cudaSuccess) return e;
  }
  trd_qform_kernel<<<kQfCtas, kTrdThreads, qf_smem, sq>>>(n, L); note_launch();
  trd_bisect_kernel<<<n, 32, 0, st>>>(n, L); note_launch();
  trd_vectors_kernel<<<ceil_div(n, kTrdEigWarps), kTrdEigWarps * 32, 0, st>>>(n, L); note_launch();
  if (fork) {
    e = cudaEventRecord(ev_q, aux);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_q, 0);
    if (e != cudaSuccess) return e;
  }
  const int tiles = ceil_div(n, 16);
  trd_gemm_kernel<0><<<dim3(tiles, tiles, 2), 256, 0, st>>>(n, L, D, Y, ldy); note_launch();
  trd_gemm_kernel<1><<<dim3(tiles, tiles, 1), 256, 0, st>>>(n, L, D, Y, ldy); note_launch();
  *run_jacobi = &L.ctl->run_jacobi;
  return cudaGetLastError();
}

}  // namespace bchdav
