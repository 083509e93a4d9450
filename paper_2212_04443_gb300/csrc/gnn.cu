// Learned start block for Algorithm 2 (an extension: the paper takes an optional V_init and
// filters it progressively, best Rayleigh quotient first, Step 17).  A three-layer
// message-passing network on the normalised adjacency Ahat = I - A proposes Z (N x k); its
// span is orthonormalised and rotated to Ritz vectors in ascending order to form V_init.
//
//   X0  = [sqrt(deg)/8, log(1 + deg)/8, R]                    R: N x d_r random features
//   S_l = (Ahat H_{l-1}) W_l + H_{l-1} U_l + 1 b_l^T,  H_l = relu(S_l),  H_0 = X0
//   Z   = H_L Wo
// Training loss against solver eigenvectors U (N x k):  G = Z^T Z + rho I,  P = U^T Z,
//   loss = 1 - tr(G^{-1} P^T P) / k  (mean sin^2 of the principal angles when rho = 0),
//   dloss/dZ = -(2/k) [U P G^{-1} - Z G^{-1} P^T P G^{-1}],  rho = ridge tr(Z^T Z) / k.
// Activations are float32 row-major N x w blocks; products with Ahat reuse the SpMM kernel
// (Ahat X = X - A X); weight gradients are Gram products over the N rows (float32 per CTA
// chunk, float64 across chunks in a fixed order: deterministic).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "handle.cuh"

namespace bchdav {
namespace {

constexpr int kGW = 64;        // widest block of the network (hidden width, k <= 64 per pass)
constexpr int kRowTile = 16;   // rows per CTA of the row products
constexpr int kGramRows = 32;  // rows staged per step of the Gram kernel

// ---- inputs
__global__ void gnn_features_kernel(int n, const int* __restrict__ rowptr,
                                    const int* __restrict__ colidx, const float* __restrict__ R,
                                    int d_r, float* __restrict__ X0) {
  const int d_in = d_r + 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int lo = rowptr[i], hi = rowptr[i + 1];
    const int len = hi - lo;
    // sorted row: binary search for the stored diagonal
    int a = lo, b = hi;
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (colidx[mid] < i) a = mid + 1;
      else b = mid;
    }
    const float deg = (float)(len - ((a < hi && colidx[a] == i) ? 1 : 0));
    X0[(size_t)i * d_in] = sqrtf(deg) * 0.125f;
    X0[(size_t)i * d_in + 1] = log1pf(deg) * 0.125f;
    for (int j = 0; j < d_r; ++j) X0[(size_t)i * d_in + 2 + j] = R[(size_t)i * d_r + j];
  }
}

// ---- row products: Y = act(a1 X1 op(W1) + a2 X2 op(W2) + bias), q <= 64 columns per pass.
// op(W) = W (p x q, row-major, ld ldw) or W^T (W stored q x p).  S (pre-activation) stored
// when non-NULL.  CTA: 16 rows x 64 columns, 256 threads, 4 rows per thread.
struct RowmmArgs {
  int n, q;
  const float* X1; int p1, ldx1; const float* W1; int ldw1; int t1; float a1;
  const float* X2; int p2, ldx2; const float* W2; int ldw2; int t2; float a2;
  const float* bias; int relu;
  float* S; float* Y; int ldy;
};

__global__ void __launch_bounds__(256) gnn_rowmm_kernel(RowmmArgs a) {
  __shared__ float sW1[kGW][kGW + 1];
  __shared__ float sW2[kGW][kGW + 1];
  __shared__ float sX1[kRowTile][kGW + 1];
  __shared__ float sX2[kRowTile][kGW + 1];
  const int t = threadIdx.x;
  const int c0 = blockIdx.y * kGW;
  const int qc = min(kGW, a.q - c0);
  const int r0 = blockIdx.x * kRowTile;
  // weights: sW[p][c] = op(W)(p, c0 + c)
  for (int idx = t; idx < kGW * kGW; idx += 256) {
    const int p = idx / kGW, c = idx % kGW;
    float w1 = 0.f, w2 = 0.f;
    if (c < qc) {
      if (p < a.p1) w1 = a.t1 ? a.W1[(size_t)(c0 + c) * a.ldw1 + p] : a.W1[(size_t)p * a.ldw1 + c0 + c];
      if (a.X2 != nullptr && p < a.p2)
        w2 = a.t2 ? a.W2[(size_t)(c0 + c) * a.ldw2 + p] : a.W2[(size_t)p * a.ldw2 + c0 + c];
    }
    sW1[p][c] = w1;
    sW2[p][c] = w2;
  }
  for (int idx = t; idx < kRowTile * kGW; idx += 256) {
    const int r = idx / kGW, p = idx % kGW;
    const int row = r0 + r;
    sX1[r][p] = (row < a.n && p < a.p1) ? a.X1[(size_t)row * a.ldx1 + p] : 0.f;
    sX2[r][p] = (a.X2 != nullptr && row < a.n && p < a.p2) ? a.X2[(size_t)row * a.ldx2 + p] : 0.f;
  }
  __syncthreads();
  constexpr int RPT = kRowTile / 4;      // rows per thread
  const int c = t % kGW, rg = t / kGW;   // 4 row groups
  if (c >= qc) return;
  float acc1[RPT], acc2[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) acc1[i] = acc2[i] = 0.f;
  for (int p = 0; p < a.p1; ++p) {
    const float w = sW1[p][c];
#pragma unroll
    for (int i = 0; i < RPT; ++i) acc1[i] = fmaf(sX1[rg * RPT + i][p], w, acc1[i]);
  }
  if (a.X2 != nullptr)
    for (int p = 0; p < a.p2; ++p) {
      const float w = sW2[p][c];
#pragma unroll
      for (int i = 0; i < RPT; ++i) acc2[i] = fmaf(sX2[rg * RPT + i][p], w, acc2[i]);
    }
  const float bc = a.bias != nullptr ? a.bias[c0 + c] : 0.f;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int row = r0 + rg * RPT + i;
    if (row >= a.n) break;
    const float s = a.a1 * acc1[i] + a.a2 * acc2[i] + bc;
    if (a.S != nullptr) a.S[(size_t)row * a.ldy + c0 + c] = s;
    a.Y[(size_t)row * a.ldy + c0 + c] = a.relu ? fmaxf(s, 0.f) : s;
  }
}

// ---- Gram products out (p x q) = X^T Y over n rows (X NULL: a column of ones, p = 1).
// CTA z sums rows [z * rows_per, (z + 1) * rows_per) in float32 into part[z] (p x q).
__global__ void __launch_bounds__(256) gnn_gram_kernel(int n, const float* __restrict__ X,
                                                       int p, int ldx, const float* __restrict__ Y,
                                                       int q, int ldy, int rows_per,
                                                       float* __restrict__ part) {
  __shared__ float sX[kGramRows][kGW + 1];
  __shared__ float sY[kGramRows][kGW + 1];
  const int t = threadIdx.x;
  const int i = t / 4, jb = (t % 4) * 16;   // output row i, columns jb .. jb + 15
  float acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.f;
  const int r_begin = blockIdx.x * rows_per;
  const int r_end = min(n, r_begin + rows_per);
  for (int r0 = r_begin; r0 < r_end; r0 += kGramRows) {
    for (int idx = t; idx < kGramRows * kGW; idx += 256) {
      const int r = idx / kGW, c = idx % kGW;
      const int row = r0 + r;
      const bool in = row < r_end;
      sX[r][c] = (in && c < p) ? (X != nullptr ? X[(size_t)row * ldx + c] : 1.f) : 0.f;
      sY[r][c] = (in && c < q) ? Y[(size_t)row * ldy + c] : 0.f;
    }
    __syncthreads();
    if (i < p)
      for (int r = 0; r < kGramRows; ++r) {
        const float x = sX[r][i];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = fmaf(x, sY[r][jb + j], acc[j]);
      }
    __syncthreads();
  }
  if (i < p)
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (jb + j < q) part[(size_t)blockIdx.x * p * q + (size_t)i * q + jb + j] = acc[j];
}

// out[i] = sum_z part[z][i] in float64, z ascending
__global__ void gnn_gram_reduce_kernel(const float* __restrict__ part, int nz, int count,
                                       double* __restrict__ out64, float* __restrict__ out32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += (double)part[(size_t)z * count + i];
    if (out64) out64[i] = s;
    if (out32) out32[i] = (float)s;
  }
}

__global__ void gnn_relu_bwd_kernel(long long total, const float* __restrict__ S,
                                    float* __restrict__ dH) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    if (!(S[i] > 0.f)) dH[i] = 0.f;
}

// ---- the k x k part of the loss (one CTA, k <= 64, float64):
// G = ZtZ + rho I = R^T R (Cholesky), K = P R^{-1}, loss = 1 - |K|_F^2 / k,
// C1 = -(2/k) K R^{-T}, C2 = (2/k) R^{-1} K^T K R^{-T}  (so dZ = U C1 + Z C2).
__global__ void __launch_bounds__(256) gnn_loss_small_kernel(int k, const double* __restrict__ P,
                                                             const double* __restrict__ ZtZ,
                                                             double ridge, double* __restrict__ loss,
                                                             float* __restrict__ C1,
                                                             float* __restrict__ C2,
                                                             int* __restrict__ flag) {
  extern __shared__ double gnn_small_smem[];
  typedef double Mat[kGW + 1];
  Mat* sR = reinterpret_cast<Mat*>(gnn_small_smem);   // G, then R (upper)
  Mat* sRi = sR + kGW;                                 // R^{-1} (upper)
  Mat* sK = sRi + kGW;                                 // K, then R^{-1} K^T K
  Mat* sT = sK + kGW;                                  // K^T K
  double* red = reinterpret_cast<double*>(sT + kGW);   // 256
  const int t = threadIdx.x;
  double tr = 0.0;
  for (int i = 0; i < k; ++i) tr += ZtZ[i * k + i];
  const double rho = ridge * tr / k;
  for (int idx = t; idx < k * k; idx += 256) {
    const int i = idx / k, j = idx % k;
    sR[i][j] = ZtZ[idx] + (i == j ? rho : 0.0);
    sRi[i][j] = 0.0;
  }
  __syncthreads();
  // right-looking Cholesky, upper factor R with G = R^T R (row i of R from column i of G)
  for (int j = 0; j < k; ++j) {
    if (t == 0) {
      const double d = sR[j][j];
      if (!(d > 0.0)) *flag = 1;
      sR[j][j] = sqrt(fmax(d, 1e-300));
    }
    __syncthreads();
    const double piv = sR[j][j];
    for (int c = j + 1 + t; c < k; c += 256) sR[j][c] /= piv;
    __syncthreads();
    for (int idx = t; idx < (k - j - 1) * (k - j - 1); idx += 256) {
      const int r = j + 1 + idx / (k - j - 1), c = j + 1 + idx % (k - j - 1);
      if (c >= r) sR[r][c] -= sR[j][r] * sR[j][c];
    }
    __syncthreads();
  }
  // R^{-1} by columns (each thread one column, back substitution)
  if (t < k) {
    const int c = t;
    for (int r = c; r >= 0; --r) {
      double s = (r == c) ? 1.0 : 0.0;
      for (int m = r + 1; m <= c; ++m) s -= sR[r][m] * sRi[m][c];
      sRi[r][c] = s / sR[r][r];
    }
  }
  __syncthreads();
  // K = P R^{-1}
  for (int idx = t; idx < k * k; idx += 256) {
    const int i = idx / k, j = idx % k;
    double s = 0.0;
    for (int m = 0; m <= j; ++m) s += P[i * k + m] * sRi[m][j];
    sK[i][j] = s;
  }
  __syncthreads();
  double part = 0.0;
  for (int idx = t; idx < k * k; idx += 256) part += sK[idx / k][idx % k] * sK[idx / k][idx % k];
  red[t] = part;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0) *loss = 1.0 - red[0] / k;
  // sT = K^T K
  for (int idx = t; idx < k * k; idx += 256) {
    const int i = idx / k, j = idx % k;
    double s = 0.0;
    for (int m = 0; m < k; ++m) s += sK[m][i] * sK[m][j];
    sT[i][j] = s;
  }
  __syncthreads();
  // C1 = -(2/k) K R^{-T}:  (K R^{-T})_ij = sum_m K_im Rinv_jm
  for (int idx = t; idx < k * k; idx += 256) {
    const int i = idx / k, j = idx % k;
    double s = 0.0;
    for (int m = j; m < k; ++m) s += sK[i][m] * sRi[j][m];
    C1[idx] = (float)(-2.0 / k * s);
  }
  __syncthreads();
  // sK <- R^{-1} (K^T K)
  for (int idx = t; idx < k * k; idx += 256) {
    const int i = idx / k, j = idx % k;
    double s = 0.0;
    for (int m = i; m < k; ++m) s += sRi[i][m] * sT[m][j];
    sK[i][j] = s;
  }
  __syncthreads();
  // C2 = (2/k) R^{-1} K^T K R^{-T}
  for (int idx = t; idx < k * k; idx += 256) {
    const int i = idx / k, j = idx % k;
    double s = 0.0;
    for (int m = j; m < k; ++m) s += sK[i][m] * sRi[j][m];
    C2[idx] = (float)(2.0 / k * s);
  }
}

__global__ void gnn_adam_kernel(int n, float* __restrict__ theta, const float* __restrict__ g,
                                float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                                float b2, float c1, float c2, float eps) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = isfinite(g[i]) ? g[i] : 0.f;   // a non-finite component is skipped
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ---------------- host side ----------------
struct Net {
  int d_in, w, k, layers;
  size_t off_W[8], off_U[8], off_b[8], off_Wo, total;
};

Net net_layout(int d_r, int w, int k) {
  Net N;
  N.d_in = d_r + 2;
  N.w = w;
  N.k = k;
  N.layers = 3;
  size_t o = 0;
  int p = N.d_in;
  for (int l = 0; l < N.layers; ++l) {
    N.off_W[l] = o;
    o += (size_t)p * w;
    N.off_U[l] = o;
    o += (size_t)p * w;
    N.off_b[l] = o;
    o += w;
    p = w;
  }
  N.off_Wo = o;
  o += (size_t)w * k;
  N.total = o;
  return N;
}

cudaError_t rowmm(cudaStream_t st, int n, int q, const float* X1, int p1, int ldx1,
                  const float* W1, int ldw1, int t1, float a1, const float* X2, int p2, int ldx2,
                  const float* W2, int ldw2, int t2, float a2, const float* bias, int relu,
                  float* S, float* Y, int ldy) {
  if (n <= 0 || q <= 0) return cudaSuccess;
  if (p1 > kGW || p2 > kGW) return cudaErrorInvalidValue;
  RowmmArgs a{n, q, X1, p1, ldx1, W1, ldw1, t1, a1, X2, p2, ldx2, W2, ldw2, t2, a2,
              bias, relu, S, Y, ldy};
  dim3 grid(ceil_div(n, kRowTile), ceil_div(q, kGW));
  gnn_rowmm_kernel<<<grid, 256, 0, st>>>(a); note_launch();
  return cudaGetLastError();
}

int gram_chunks(int n) { return std::max(1, std::min(4 * kSMs, ceil_div(n, 1024))); }

// out64 / out32 (p x q) = X^T Y; part holds gram_chunks(n) * p * q floats
cudaError_t gram(cudaStream_t st, int n, const float* X, int p, int ldx, const float* Y, int q,
                 int ldy, float* part, double* out64, float* out32) {
  if (p > kGW || q > kGW) return cudaErrorInvalidValue;
  const int nz = gram_chunks(n);
  const int rows_per = ceil_div(n, nz);
  gnn_gram_kernel<<<nz, 256, 0, st>>>(n, X, p, ldx, Y, q, ldy, rows_per, part); note_launch();
  gnn_gram_reduce_kernel<<<ceil_div(p * q, 256), 256, 0, st>>>(part, nz, p * q, out64, out32);
  note_launch();
  return cudaGetLastError();
}

}  // namespace
}  // namespace bchdav

using namespace bchdav;

#define HCUDA(expr) BCHDAV_CUDA_OK(expr, h)

namespace {

// workspace of one network pass over a graph with n nodes (float32 blocks)
struct GnnWork {
  float* X0;       // n x d_in
  float* H[4];     // H_0 = X0, H_1..H_3 (n x w)
  float* AH[3];    // Ahat H_{l-1}
  float* S[3];     // pre-activations
  float* Z;        // n x k
  float* U32;      // n x k targets
  float* dZ;       // n x k
  float* dH;       // n x w
  float* T;        // n x w
  float* Q;        // n x w
  float* part;     // gram partials
  double* small;   // P, ZtZ (k x k each) + loss
  float* C;        // C1, C2 (k x k each)
  int* flag;
};

size_t gnn_work_bytes(int n, const Net& N, bool train) {
  const size_t nw = (size_t)n * N.w, nk = (size_t)n * N.k, nd = (size_t)n * N.d_in;
  size_t f = nd + (train ? 3 * nw + 3 * nw + 3 * nw : 2 * nw + nw + nw) + nk;
  if (train) f += 2 * nk + 3 * nw;
  f += (size_t)gram_chunks(n) * kGW * kGW;
  return f * sizeof(float) + (2 * kGW * kGW + 16) * sizeof(double) + 2 * kGW * kGW * sizeof(float) +
         4096;
}

GnnWork carve(void* base, int n, const Net& N, bool train) {
  GnnWork w;
  std::memset(&w, 0, sizeof(w));
  char* p = static_cast<char*>(base);
  auto take = [&](size_t floats) {
    float* r = reinterpret_cast<float*>(p);
    p += ((floats * sizeof(float) + 255) / 256) * 256;
    return r;
  };
  const size_t nw = (size_t)n * N.w, nk = (size_t)n * N.k;
  w.X0 = take((size_t)n * N.d_in);
  w.H[0] = w.X0;
  if (train) {
    for (int l = 1; l <= 3; ++l) w.H[l] = take(nw);
    for (int l = 0; l < 3; ++l) w.AH[l] = take(nw);
    for (int l = 0; l < 3; ++l) w.S[l] = take(nw);
  } else {
    // inference keeps two ping-pong activations and one Ahat H buffer
    float* a = take(nw);
    float* b = take(nw);
    w.H[1] = a;
    w.H[2] = b;
    w.H[3] = a;
    float* ah = take(nw);
    w.AH[0] = w.AH[1] = w.AH[2] = ah;
  }
  w.Z = take(nk);
  if (train) {
    w.U32 = take(nk);
    w.dZ = take(nk);
    w.dH = take(nw);
    w.T = take(nw);
    w.Q = take(nw);
  }
  w.part = take((size_t)gram_chunks(n) * kGW * kGW);
  w.small = reinterpret_cast<double*>(p);
  p += (2 * kGW * kGW + 16) * sizeof(double);
  w.C = take(2 * kGW * kGW);
  w.flag = reinterpret_cast<int*>(p);
  return w;
}

bchdav_status check_net_args(bchdav_handle h, const bchdav_csr* A, int d_r, int w, int k) {
  if (!A || A->n <= 0 || !A->rowptr || !A->colidx || !A->val_f32) {
    h->set_error(BCHDAV_ERR_ARG, "gnn: CSR with float32 values required");
    return BCHDAV_ERR_ARG;
  }
  if (d_r < 0 || d_r + 2 > kGW || w < 1 || w > kGW || k < 1 || k > kGW || (w % 4) != 0 ||
      ((d_r + 2) % 4) != 0) {
    h->set_error(BCHDAV_ERR_ARG,
                 "gnn: need d_r + 2 and width multiples of 4, at most 64; 1 <= k <= 64");
    return BCHDAV_ERR_ARG;
  }
  return BCHDAV_OK;
}

// Ahat X = X - A X  (X: n x p, p multiple of 4)
cudaError_t ahat(cudaStream_t st, const bchdav_csr* A, const float* X, int p, float* Y,
                 const float* Zadd = nullptr, const SpmmLong* lg = nullptr) {
  return launch_spmm_axpby<float>(st, A->n, A->rowptr, A->colidx, A->val_f32, X, p, p, Y, p, Zadd,
                                  p, -1.f, 1.f, Zadd ? 1.f : 0.f, nullptr, 0, nullptr, lg);
}

bchdav_status forward(bchdav_handle h, const bchdav_csr* A, const float* R, const Net& N,
                      const float* theta, GnnWork& w, bool keep) {
  cudaStream_t st = h->stream;
  const int n = A->n;
  gnn_features_kernel<<<std::min(ceil_div(n, 256), 16 * kSMs), 256, 0, st>>>(
      n, A->rowptr, A->colidx, R, N.d_in - 2, w.X0); note_launch();
  int p = N.d_in;
  for (int l = 0; l < N.layers; ++l) {
    HCUDA(ahat(st, A, w.H[l], p, w.AH[l], nullptr, h->long_rows()));
    HCUDA(rowmm(st, n, N.w, w.AH[l], p, p, theta + N.off_W[l], N.w, 0, 1.f, w.H[l], p, p,
                theta + N.off_U[l], N.w, 0, 1.f, theta + N.off_b[l], 1, keep ? w.S[l] : nullptr,
                w.H[l + 1], N.w));
    p = N.w;
  }
  HCUDA(rowmm(st, n, N.k, w.H[N.layers], N.w, N.w, theta + N.off_Wo, N.k, 0, 1.f, nullptr, 0, 0,
              nullptr, 0, 0, 0.f, nullptr, 0, nullptr, w.Z, N.k));
  return BCHDAV_OK;
}

// loss and gradient of one graph; grad (N.total floats) is overwritten
bchdav_status loss_grad(bchdav_handle h, const bchdav_csr* A, const float* R, const Net& N,
                        const float* theta, const double* U, double ridge, float* grad,
                        GnnWork& w, double* loss_dev) {
  cudaStream_t st = h->stream;
  const int n = A->n, k = N.k;
  BCHDAV_TRY(forward(h, A, R, N, theta, w, true));
  HCUDA(launch_f64_to_f32(st, n, k, U, k, w.U32, k));
  double* P = w.small;
  double* ZtZ = w.small + kGW * kGW;
  HCUDA(gram(st, n, w.U32, k, k, w.Z, k, k, w.part, P, nullptr));
  HCUDA(gram(st, n, w.Z, k, k, w.Z, k, k, w.part, ZtZ, nullptr));
  float* C1 = w.C;
  float* C2 = w.C + kGW * kGW;
  {
    const size_t smem = (4 * kGW * (kGW + 1) + 256) * sizeof(double);
    static const cudaError_t attr = cudaFuncSetAttribute(
        gnn_loss_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    HCUDA(attr);
    gnn_loss_small_kernel<<<1, 256, smem, st>>>(k, P, ZtZ, ridge, loss_dev, C1, C2, w.flag);
    note_launch();
  }
  // dZ = U C1 + Z C2
  HCUDA(rowmm(st, n, k, w.U32, k, k, C1, k, 0, 1.f, w.Z, k, k, C2, k, 0, 1.f, nullptr, 0, nullptr,
              w.dZ, k));
  // output layer
  const int L = N.layers;
  HCUDA(gram(st, n, w.H[L], N.w, N.w, w.dZ, k, k, w.part, nullptr, grad + N.off_Wo));
  HCUDA(rowmm(st, n, N.w, w.dZ, k, k, theta + N.off_Wo, k, 1, 1.f, nullptr, 0, 0, nullptr, 0, 0,
              0.f, nullptr, 0, nullptr, w.dH, N.w));
  for (int l = L - 1; l >= 0; --l) {
    const int p = l == 0 ? N.d_in : N.w;
    const long long tot = (long long)n * N.w;
    gnn_relu_bwd_kernel<<<(int)std::min<long long>(ceil_div(tot, 256LL), 16 * kSMs), 256, 0, st>>>(
        tot, w.S[l], w.dH); note_launch();
    HCUDA(gram(st, n, w.AH[l], p, p, w.dH, N.w, N.w, w.part, nullptr, grad + N.off_W[l]));
    HCUDA(gram(st, n, w.H[l], p, p, w.dH, N.w, N.w, w.part, nullptr, grad + N.off_U[l]));
    HCUDA(gram(st, n, nullptr, 1, 0, w.dH, N.w, N.w, w.part, nullptr, grad + N.off_b[l]));
    if (l > 0) {
      // dH_{l-1} = Ahat (dS W^T) + dS U^T
      HCUDA(rowmm(st, n, p, w.dH, N.w, N.w, theta + N.off_W[l], N.w, 1, 1.f, nullptr, 0, 0,
                  nullptr, 0, 0, 0.f, nullptr, 0, nullptr, w.T, p));
      HCUDA(rowmm(st, n, p, w.dH, N.w, N.w, theta + N.off_U[l], N.w, 1, 1.f, nullptr, 0, 0,
                  nullptr, 0, 0, 0.f, nullptr, 0, nullptr, w.Q, p));
      HCUDA(ahat(st, A, w.T, p, w.dH, w.Q, h->long_rows()));
    }
  }
  return BCHDAV_OK;
}

}  // namespace

extern "C" {

int64_t bchdav_gnn_n_params(int32_t d_r, int32_t width, int32_t k) {
  if (d_r < 0 || width < 1 || k < 1) return -1;
  return (int64_t)net_layout(d_r, width, k).total;
}

bchdav_status bchdav_gnn_forward(bchdav_handle h, const bchdav_csr* A, const float* R, int32_t d_r,
                                 const float* theta, int32_t width, int32_t k, float* Z) {
  if (!h) return BCHDAV_ERR_ARG;
  BCHDAV_TRY(check_net_args(h, A, d_r, width, k));
  if (!R || !theta || !Z) return BCHDAV_ERR_ARG;
  const Net N = net_layout(d_r, width, k);
  BCHDAV_TRY(prepare_long_rows(h, A, (size_t)kGW * sizeof(float)));
  BCHDAV_TRY(h->ensure(h->gnn, gnn_work_bytes(A->n, N, false)));
  GnnWork w = carve(h->gnn.p, A->n, N, false);
  BCHDAV_TRY(forward(h, A, R, N, theta, w, false));
  HCUDA(cudaMemcpyAsync(Z, w.Z, (size_t)A->n * k * sizeof(float), cudaMemcpyDeviceToDevice,
                        h->stream));
  return BCHDAV_OK;
}

bchdav_status bchdav_gnn_loss_grad(bchdav_handle h, const bchdav_csr* A, const float* R,
                                   int32_t d_r, const float* theta, int32_t width, int32_t k,
                                   const double* U, double ridge, float* grad, double* loss,
                                   float* Z) {
  if (!h) return BCHDAV_ERR_ARG;
  BCHDAV_TRY(check_net_args(h, A, d_r, width, k));
  if (!R || !theta || !U || !grad || !loss || !(ridge >= 0)) return BCHDAV_ERR_ARG;
  const Net N = net_layout(d_r, width, k);
  BCHDAV_TRY(prepare_long_rows(h, A, (size_t)kGW * sizeof(float)));
  BCHDAV_TRY(h->ensure(h->gnn, gnn_work_bytes(A->n, N, true)));
  GnnWork w = carve(h->gnn.p, A->n, N, true);
  double* loss_dev = w.small + 2 * kGW * kGW;
  BCHDAV_TRY(loss_grad(h, A, R, N, theta, U, ridge, grad, w, loss_dev));
  HCUDA(cudaMemcpyAsync(loss, loss_dev, sizeof(double), cudaMemcpyDefault, h->stream));
  if (Z)
    HCUDA(cudaMemcpyAsync(Z, w.Z, (size_t)A->n * k * sizeof(float), cudaMemcpyDeviceToDevice,
                          h->stream));
  HCUDA(cudaStreamSynchronize(h->stream));
  return BCHDAV_OK;
}

bchdav_status bchdav_gnn_start_block(bchdav_handle h, const bchdav_csr* A, const float* R,
                                     int32_t d_r, const float* theta, int32_t width, int32_t k,
                                     double* V0, double* ritz) {
  if (!h) return BCHDAV_ERR_ARG;
  BCHDAV_TRY(check_net_args(h, A, d_r, width, k));
  if (!R || !theta || !V0 || !ritz || !A->val || k > A->n) return BCHDAV_ERR_ARG;
  const Net N = net_layout(d_r, width, k);
  const int n = A->n;
  cudaStream_t st = h->stream;
  BCHDAV_TRY(prepare_long_rows(h, A, (size_t)kGW * sizeof(double)));
  BCHDAV_TRY(h->ensure(h->gnn, gnn_work_bytes(n, N, false)));
  GnnWork w = carve(h->gnn.p, n, N, false);
  BCHDAV_TRY(forward(h, A, R, N, theta, w, false));
  HCUDA(launch_f32_to_f64(st, n, k, w.Z, k, V0, k));
  // orthonormal basis of span(Z) (dependent columns replaced by random ones)
  int64_t rep = 0;
  int32_t nrep = 0;
  BCHDAV_TRY(bchdav_orthonormalize(h, n, nullptr, k, 0, V0, k, k, 0x5eedULL, 1e-10, &rep, &nrep));
  // Rayleigh-Ritz on the block: Hq = V0^T A V0, Hq Y = Y D, V0 <- V0 Y (ascending D)
  BCHDAV_TRY(h->ensure(h->gnn_w, ((size_t)n * k + 3 * (size_t)k * k) * sizeof(double)));
  double* AV = h->gnn_w.as<double>();
  double* Hq = AV + (size_t)n * k;
  double* Y = Hq + (size_t)k * k;
  BCHDAV_TRY(bchdav_spmm(h, A, V0, k, k, AV, k));
  BCHDAV_TRY(bchdav_gram(h, n, V0, k, k, AV, k, k, Hq, 1));
  BCHDAV_TRY(bchdav_eigh(h, k, Hq, k, ritz, Y, k));
  BCHDAV_TRY(bchdav_rotate(h, n, V0, k, k, Y, k, k, 0));
  HCUDA(cudaStreamSynchronize(st));
  // one-shot N-sized buffers: give the memory back to the solve that follows
  h->gnn.release();
  h->gnn_w.release();
  return BCHDAV_OK;
}

bchdav_status bchdav_gnn_train(bchdav_handle h, int32_t n_graphs, const bchdav_csr* As,
                               const float* const* R, int32_t d_r, const double* const* U,
                               int32_t width, int32_t k, float* theta, int32_t steps, double lr,
                               double ridge, double* loss_history) {
  if (!h || n_graphs < 1 || !As || !R || !U || !theta || steps < 0 || !(lr > 0) ||
      !(ridge >= 0))
    return BCHDAV_ERR_ARG;
  const Net N = net_layout(d_r, width, k);
  int n_max = 0;
  for (int g = 0; g < n_graphs; ++g) {
    BCHDAV_TRY(check_net_args(h, &As[g], d_r, width, k));
    n_max = std::max(n_max, As[g].n);
  }
  cudaStream_t st = h->stream;
  BCHDAV_TRY(h->ensure(h->gnn, gnn_work_bytes(n_max, N, true)));
  BCHDAV_TRY(h->ensure(h->gnn_opt, (3 * N.total + 64) * sizeof(float) + 64 * sizeof(double)));
  float* grad = h->gnn_opt.as<float>();
  float* m = grad + N.total;
  float* v = m + N.total;
  double* losses = reinterpret_cast<double*>(h->gnn_opt.as<char>() + (3 * N.total + 64) * sizeof(float));
  HCUDA(cudaMemsetAsync(m, 0, 2 * N.total * sizeof(float), st));
  const float b1 = 0.9f, b2 = 0.999f;
  int t = 0;
  for (int s = 0; s < steps; ++s) {
    for (int g = 0; g < n_graphs; ++g) {
      // the long-row schedule and workspace follow the graph
      BCHDAV_TRY(prepare_long_rows(h, &As[g], (size_t)kGW * sizeof(float)));
      GnnWork w = carve(h->gnn.p, As[g].n, N, true);
      BCHDAV_TRY(loss_grad(h, &As[g], R[g], N, theta, U[g], ridge, grad, w, losses + (g % 64)));
      ++t;
      const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
      gnn_adam_kernel<<<std::min(ceil_div((int)N.total, 256), 4 * kSMs), 256, 0, st>>>(
          (int)N.total, theta, grad, m, v, (float)lr, b1, b2, c1, c2, 1e-8f); note_launch();
      if (loss_history) {
        HCUDA(cudaMemcpyAsync(loss_history + (size_t)s * n_graphs + g, losses + (g % 64),
                              sizeof(double), cudaMemcpyDefault, st));
      }
    }
  }
  HCUDA(cudaStreamSynchronize(st));
  return BCHDAV_OK;
}

}  // extern "C"
