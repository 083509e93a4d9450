// C-ABI entry points and the device-resident driver of Algorithm 2 (block
// Chebyshev-Davidson with inner-outer restart).  Every vector and matrix of
// the iteration lives in device memory; per outer iteration the host reads
// back only the k_act Ritz values and the k_b residual norms it needs for the
// control decisions of Steps 10-18.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "handle.cuh"
#include "kernels.cuh"

using namespace bchdav;

namespace {

// Message for entry points without a handle; one per host thread, so that calls made at the
// same time from different threads (e.g. on different devices) never share the string.
thread_local std::string g_create_error;

constexpr double kTauDepF64 = 1e-10;
constexpr double kTauDepMixed = 1e-10;
constexpr double kLowNwbEps = 1e-12;
// Mixed path: digit slices of the product that a later float64-accurate step repairs (the first
// DGKS projection, whose error lies in span(V) and is removed by the second).  4 slices keep 24
// bits of each operand.
constexpr int kMixedPass1Slices = 4;

#define HCUDA(expr) BCHDAV_CUDA_OK(expr, h)

bchdav_status check_csr_args(bchdav_handle h, const bchdav_csr* A) {
  if (!A || A->n <= 0 || !A->rowptr || !A->colidx || !A->val || A->nnz < A->n ||
      A->nnz >= (int64_t)INT32_MAX) {
    h->set_error(BCHDAV_ERR_ARG, "invalid CSR descriptor");
    return BCHDAV_ERR_ARG;
  }
  return BCHDAV_OK;
}

// ---------------- timing helper ----------------
struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  double acc = 0.0;
  bool pending = false;
  void init() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  void destroy() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  void start(cudaStream_t s) { cudaEventRecord(a, s); }
  void stop(cudaStream_t s) {
    cudaEventRecord(b, s);
    pending = true;
  }
  void collect() {   // after a stream sync
    if (!pending) return;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess) acc += ms;
    pending = false;
  }
};

// Filter SpMM schedule: the row kernel's block size (rows per CTA) for a matrix and block width.
// Small graphs want small blocks (enough CTAs to cover the GPU); large ones fewer, larger blocks.
// The choice is made by timing each candidate on the first filter step's own buffers (every
// candidate computes every row the same way, so the choice never changes a result) and kept at
// two levels: per matrix in the handle, and in a process-wide table keyed on the matrix's
// class -- N and the mean row length in half-octaves, the block width, the value size, and
// whether long rows are split into segments (the degree skew the row kernel sees) -- so that
// later matrices of the same class (the graphs of a batch, the next solve) take the entry
// without timing.  Vector width and the long-row split follow from the block width, alignment
// and row lengths (spmm.cu).
struct SpmmClass {
  int logn2, deg2, b, vsize, skew;
  bool operator==(const SpmmClass& o) const {
    return logn2 == o.logn2 && deg2 == o.deg2 && b == o.b && vsize == o.vsize && skew == o.skew;
  }
};
std::mutex g_spmm_class_mu;
std::vector<std::pair<SpmmClass, int>> g_spmm_class_table;

SpmmClass spmm_class(const bchdav_csr* A, int b, int vsize, bool long_rows) {
  SpmmClass c;
  const double n = std::max(1, A->n);
  c.logn2 = (int)std::floor(2.0 * std::log2(n));
  c.deg2 = (int)std::floor(2.0 * std::log2(std::max(1.0, (double)A->nnz / n)));
  c.b = b;
  c.vsize = vsize;
  c.skew = long_rows ? 1 : 0;
  return c;
}

template <typename F>
bchdav_status spmm_schedule(bchdav_handle h, const bchdav_csr* A, int b, int vsize, F run,
                            int* threads) {
  for (const auto& e : h->spmm_tune)
    if (e.rowptr == A->rowptr && e.n == A->n && e.nnz == A->nnz && e.b == b && e.vsize == vsize) {
      *threads = e.threads;
      return BCHDAV_OK;
    }
  const SpmmClass cls = spmm_class(A, b, vsize, h->lg.n_seg > 0);
  {
    std::lock_guard<std::mutex> lk(g_spmm_class_mu);
    for (const auto& e : g_spmm_class_table)
      if (e.first == cls) {
        *threads = e.second;
        h->spmm_tune.push_back({A->rowptr, A->n, A->nnz, b, vsize, e.second});
        return BCHDAV_OK;
      }
  }
  cudaStream_t st = h->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HCUDA(cudaEventCreate(&e0));
  HCUDA(cudaEventCreate(&e1));
  const int cand[4] = {64, 128, 256, 512};
  float best = 3.0e38f;
  int best_t = 256;
  cudaError_t err = cudaSuccess;
  for (int c : cand) {
    if ((err = run(c)) != cudaSuccess) break;   // warm
    if ((err = cudaEventRecord(e0, st)) != cudaSuccess) break;
    if ((err = run(c)) != cudaSuccess || (err = run(c)) != cudaSuccess) break;
    if ((err = cudaEventRecord(e1, st)) != cudaSuccess) break;
    if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    if ((err = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
    if (ms < best) {
      best = ms;
      best_t = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HCUDA(err);
  h->spmm_tune.push_back({A->rowptr, A->n, A->nnz, b, vsize, best_t});
  {
    std::lock_guard<std::mutex> lk(g_spmm_class_mu);
    bool found = false;
    for (const auto& e : g_spmm_class_table) found = found || e.first == cls;
    if (!found) g_spmm_class_table.push_back({cls, best_t});
  }
  *threads = best_t;
  return BCHDAV_OK;
}

// ---------------- Algorithm 3 ----------------
// Y = p_m(A) X.  prec MIXED: recurrence in float32 (val32 required).
bchdav_status run_filter(bchdav_handle h, const bchdav_csr* A, const float* val32, const double* X,
                         int ldx, int b, int m, double a, double upb, double a0, int prec,
                         double* Y, int ldy, double* bytes_out) {
  const int n = A->n;
  cudaStream_t st = h->stream;
  const double c = (a + upb) / 2.0, e = (upb - a) / 2.0;
  double sigma = e / (a0 - c);
  const double tau = 2.0 / sigma;
  const size_t sx = prec == BCHDAV_PREC_MIXED ? 4 : 8;
  const int ldb = prec == BCHDAV_PREC_MIXED ? round_up(b, 4) : round_up(b, 2);
  for (int i = 0; i < 4; ++i) BCHDAV_TRY(h->ensure(h->F[i], (size_t)n * ldb * sx));
  double bytes = 0.0;
  const double csr_bytes = 4.0 * (n + 1) + (double)A->nnz * (4.0 + (double)sx);
  if (prec == BCHDAV_PREC_MIXED) {
    float* T[4] = {h->F[0].as<float>(), h->F[1].as<float>(), h->F[2].as<float>(),
                   h->F[3].as<float>()};
    HCUDA(launch_f64_to_f32(st, n, b, X, ldx, T[0], ldb));
    int thr = 256;
    BCHDAV_TRY(spmm_schedule(h, A, b, 4, [&](int bs) {
      return launch_spmm_axpby<float>(st, n, A->rowptr, A->colidx, val32, T[0], ldb, b, T[1], ldb,
                                      nullptr, 0, 1.f, 0.f, 0.f, nullptr, 0, nullptr,
                                      h->long_rows(), bs);
    }, &thr));
    // step 1: U = (A X - c X) sigma / e
    HCUDA(launch_spmm_axpby<float>(st, n, A->rowptr, A->colidx, val32, T[0], ldb, b, T[1], ldb,
                                   nullptr, 0, (float)(sigma / e), (float)(-c * sigma / e), 0.f,
                                   nullptr, 0, nullptr, h->long_rows(), thr));
    bytes += csr_bytes + 3.0 * n * b * sx;
    int prev = 0, cur = 1;
    for (int i = 2; i <= m; ++i) {
      double sigma1 = 1.0 / (tau - sigma);
      int nxt = 0;
      while (nxt == prev || nxt == cur) ++nxt;
      HCUDA(launch_spmm_axpby<float>(st, n, A->rowptr, A->colidx, val32, T[cur], ldb, b, T[nxt],
                                     ldb, T[prev], ldb, (float)(2.0 * sigma1 / e),
                                     (float)(-2.0 * sigma1 * c / e), (float)(-sigma * sigma1),
                                     nullptr, 0, nullptr, h->long_rows(), thr));
      bytes += csr_bytes + 4.0 * n * b * sx;
      prev = cur;
      cur = nxt;
      sigma = sigma1;
    }
    HCUDA(launch_f32_to_f64(st, n, b, T[cur], ldb, Y, ldy));
  } else {
    double* T[4] = {h->F[0].as<double>(), h->F[1].as<double>(), h->F[2].as<double>(),
                    h->F[3].as<double>()};
    const double* prevp = X;
    int prevld = ldx;
    double* out = (m == 1) ? Y : T[0];
    int outld = (m == 1) ? ldy : ldb;
    int thr = 256;
    BCHDAV_TRY(spmm_schedule(h, A, b, 8, [&](int bs) {
      return launch_spmm_axpby<double>(st, n, A->rowptr, A->colidx, A->val, X, ldx, b, T[1], ldb,
                                       nullptr, 0, 1.0, 0.0, 0.0, nullptr, 0, nullptr,
                                       h->long_rows(), bs);
    }, &thr));
    HCUDA(launch_spmm_axpby<double>(st, n, A->rowptr, A->colidx, A->val, X, ldx, b, out, outld,
                                    nullptr, 0, sigma / e, -c * sigma / e, 0.0, nullptr, 0, nullptr,
                                    h->long_rows(), thr));
    bytes += csr_bytes + 3.0 * n * b * sx;
    const double* curp = out;
    int curld = outld;
    int slot = 1;
    for (int i = 2; i <= m; ++i) {
      double sigma1 = 1.0 / (tau - sigma);
      double* nxt;
      int nxtld;
      if (i == m) {
        nxt = Y;
        nxtld = ldy;
      } else {
        nxt = T[slot % 3];
        nxtld = ldb;
        ++slot;
      }
      HCUDA(launch_spmm_axpby<double>(st, n, A->rowptr, A->colidx, A->val, curp, curld, b, nxt,
                                      nxtld, prevp, prevld, 2.0 * sigma1 / e,
                                      -2.0 * sigma1 * c / e, -sigma * sigma1, nullptr, 0, nullptr,
                                      h->long_rows(), thr));
      bytes += csr_bytes + 4.0 * n * b * sx;
      prevp = curp;
      prevld = curld;
      curp = nxt;
      curld = nxtld;
      sigma = sigma1;
    }
  }
  if (bytes_out) *bytes_out += bytes;
  return BCHDAV_OK;
}

// Mixed-precision filter of Step 5.  Column j is either a plain column
// (theta[j] is NaN): float32 recurrence of Algorithm 3 on X(:, j); or the
// residual r_j = A u_j - theta_j u_j of a Ritz pair (theta_j finite): the
// float32 recurrence applies s(x) = (p(x) - p(theta_j)) / (x - theta_j) to r_j,
//   Z_1 = (sigma_1 / e) r,
//   Z_{k+1} = (2 sigma_{k+1} / e) ((A - c) Z_k + p_k(theta) r) - sigma_k sigma_{k+1} Z_{k-1},
// since p(A) u_j = p(theta_j) u_j + s(A) r_j with u_j in the basis, both give
// the same vector after orthogonalisation against the basis (Step 6), and the
// float32 rounding is relative to ||s(A) r_j|| instead of ||p(A) u_j||.
bchdav_status run_filter_mixed(bchdav_handle h, const bchdav_csr* A, const float* val32,
                               const double* X, int ldx, const double* R, int ldr,
                               const int* src_host, const double* theta, int b, int m, double a,
                               double upb, double a0, double* Y, int ldy, double* bytes_out) {
  const int n = A->n;
  cudaStream_t st = h->stream;
  const double c = (a + upb) / 2.0, e = (upb - a) / 2.0;
  const double sigma1 = e / (a0 - c);
  const double tau = 2.0 / sigma1;
  const int ldb = round_up(b, 4);
  for (int i = 0; i < 4; ++i) BCHDAV_TRY(h->ensure(h->F[i], (size_t)n * ldb * sizeof(float)));
  float* T[4] = {h->F[0].as<float>(), h->F[1].as<float>(), h->F[2].as<float>(),
                 h->F[3].as<float>()};
  // R32 lives in the fourth float buffer's twin: reuse mix buffer for coefficients
  BCHDAV_TRY(h->ensure(h->mix, (size_t)(m + 1) * 64 * sizeof(float) + 64 * sizeof(int) +
                                   (size_t)n * ldb * sizeof(float) + 256));
  int* src_d = reinterpret_cast<int*>(h->mix.p);
  float* delta_d = reinterpret_cast<float*>(h->mix.as<char>() + 64 * sizeof(int));
  float* R32 = reinterpret_cast<float*>(
      h->mix.as<char>() + 64 * sizeof(int) + (size_t)(m + 1) * 64 * sizeof(float));
  // host: sigma sequence, p_k(theta_j), deltas
  BCHDAV_TRY(h->ensure_aux((size_t)(m + 1) * 64 + 128));
  HCUDA(cudaStreamSynchronize(st));   // earlier copies from host_aux are complete
  float* dh = reinterpret_cast<float*>(h->host_aux);
  int* sh = reinterpret_cast<int*>(h->host_aux + (size_t)(m + 1) * 32 + 32);
  bool any_res = false;
  std::vector<double> pkm1(b, 1.0), pk(b, 0.0);
  for (int j = 0; j < b; ++j) {
    bool res = src_host[j] >= 0;
    any_res = any_res || res;
    sh[j] = src_host[j];
    pk[j] = res ? sigma1 * (theta[j] - c) / e : 0.0;   // p_1(theta)
    dh[j] = res ? (float)(sigma1 / e) : 0.f;            // step 1 coefficient
  }
  std::vector<double> sig(m + 1);
  sig[1] = sigma1;
  for (int i = 2; i <= m; ++i) {
    sig[i] = 1.0 / (tau - sig[i - 1]);
    for (int j = 0; j < b; ++j) {
      bool res = src_host[j] >= 0;
      // coefficient of r in step i uses p_{i-1}(theta)
      dh[(size_t)(i - 1) * 64 + j] = res ? (float)(2.0 * sig[i] / e * pk[j]) : 0.f;
      double pnew = res ? (2.0 * sig[i] / e * (theta[j] - c) * pk[j] - sig[i - 1] * sig[i] * pkm1[j])
                        : 0.0;
      pkm1[j] = pk[j];
      pk[j] = pnew;
    }
  }
  HCUDA(cudaMemcpyAsync(src_d, sh, b * sizeof(int), cudaMemcpyHostToDevice, st));
  HCUDA(cudaMemcpyAsync(delta_d, dh, (size_t)m * 64 * sizeof(float), cudaMemcpyHostToDevice, st));
  HCUDA(launch_mixed_inputs(st, n, b, X, ldx, any_res ? R : X, any_res ? ldr : ldx, src_d, T[0],
                            R32, ldb));
  const float* Rp = any_res ? R32 : nullptr;
  int thr = 256;
  BCHDAV_TRY(spmm_schedule(h, A, b, 4, [&](int bs) {
    return launch_spmm_axpby<float>(st, n, A->rowptr, A->colidx, val32, T[0], ldb, b, T[1], ldb,
                                    nullptr, 0, 1.f, 0.f, 0.f, nullptr, 0, nullptr,
                                    h->long_rows(), bs);
  }, &thr));
  const double csr_bytes = 4.0 * (n + 1) + (double)A->nnz * 8.0;
  double bytes = 0.0;
  HCUDA(launch_spmm_axpby<float>(st, n, A->rowptr, A->colidx, val32, T[0], ldb, b, T[1], ldb,
                                 nullptr, 0, (float)(sigma1 / e), (float)(-c * sigma1 / e), 0.f, Rp,
                                 ldb, delta_d, h->long_rows(), thr));
  bytes += csr_bytes + (any_res ? 4.0 : 3.0) * n * b * 4.0;
  int prev = 0, cur = 1;
  for (int i = 2; i <= m; ++i) {
    int nxt = 0;
    while (nxt == prev || nxt == cur) ++nxt;
    HCUDA(launch_spmm_axpby<float>(st, n, A->rowptr, A->colidx, val32, T[cur], ldb, b, T[nxt], ldb,
                                   T[prev], ldb, (float)(2.0 * sig[i] / e),
                                   (float)(-2.0 * sig[i] * c / e), (float)(-sig[i - 1] * sig[i]),
                                   Rp, ldb, delta_d + (size_t)(i - 1) * 64, h->long_rows(), thr));
    bytes += csr_bytes + (any_res ? 5.0 : 4.0) * n * b * 4.0;
    prev = cur;
    cur = nxt;
  }
  HCUDA(launch_f32_to_f64(st, n, b, T[cur], ldb, Y, ldy));
  if (bytes_out) *bytes_out += bytes;
  return BCHDAV_OK;
}

// Gram product A^T B of cached transposed planes (Steps 6 and 8): on tcgen05 with tensor-memory
// level sums (dense_path 0) or on warp-level mma (dense_path 2); partial sums in oz_part.
cudaError_t gram_planes(bchdav_handle h, int dense_path, int Np, const void* PA, const int* EA,
                        int capA, int a0, int ka, const void* PB, const int* EB, int capB, int kb,
                        double* out, int slices = 8) {
  if (dense_path == 0)
    return launch_tc_gram(h->stream, Np, PA, EA, capA, a0, ka, PB, EB, capB, kb, out,
                          h->oz_part.as<double>(), slices, h->tc_err.as<int>());
  return oz_gram_from_planes(h->stream, Np, PA, EA, capA, a0, ka, PB, EB, capB, kb, out,
                             h->oz_part.as<double>(), slices);
}

// ---------------- Step 6 ----------------
// Where the cached slices of V live: column planes of V (S x capV x Np, exponents after them) in
// oz_vt and row planes (S x n x KpCap, exponents after them) in oz_vr.  Both are sized for the
// largest subspace `cols` once, so that the exponent arrays stay at fixed offsets for every call.
// KpCap is at least 64: the row planes' buffer also takes the block's own row planes (b <= 64
// columns) for the CholQR step of Step 6.
struct OzLayout {
  int Np, capV, KpCap;
  size_t vt_planes, vr_planes;
};
OzLayout oz_layout(int n, int cols) {
  OzLayout L;
  cols = std::max(cols, 1);
  L.Np = oz_pad_k(n);
  L.capV = oz_pad_rows(cols);
  L.KpCap = oz_pad_k(std::max(cols, 64));
  L.vt_planes = oz_planes_bytes(L.capV, L.Np);
  L.vr_planes = oz_planes_bytes(n, L.KpCap);
  return L;
}

// cap_cols: number of V columns the cached planes must be able to hold (0: just k).
// vt_valid (optional): on return, the number of leading columns of V whose column planes are
// current in oz_vt (k when this call made them, else 0).
// pass1_slices: digit slices of the first projection's Gram product V^T X (8: float64-accurate;
// 4 on the mixed path: operands to 24 bits, a TF32x3-class product).  Its error lies in span(V),
// which the second, float64-accurate pass removes; the update X -= V C always uses all of V's
// slices (a truncated V would leave error outside span(V)).
bchdav_status run_orth(bchdav_handle h, int n, const double* V, int ldv, int k, double* X, int ldx,
                       int b, uint64_t seed, double tau_dep, int64_t* rep_counter, int* n_rep,
                       int dense_path = 0, int cap_cols = 0, int* vt_valid = nullptr,
                       int pass1_slices = 8) {
  cudaStream_t st = h->stream;
  if (b > 64) {
    h->set_error(BCHDAV_ERR_ARG, "block size b must be <= 64");
    return BCHDAV_ERR_ARG;
  }
  const int chunks = gemm_tn_chunks(n);
  const int ka_max = std::max(k, 1);
  const size_t part_doubles = (size_t)chunks * std::max(ka_max, b) * b;
  BCHDAV_TRY(h->ensure(h->part, part_doubles * sizeof(double)));
  const size_t g_words = (size_t)std::max(ka_max * b, 64 * 64);
  BCHDAV_TRY(h->ensure(h->G, (g_words + 64 * 64 + 8 + 64 + 16) * sizeof(double)));
  BCHDAV_TRY(h->ensure(h->norm0, (size_t)(3 * 64 + 16) * sizeof(double)));
  BCHDAV_TRY(h->ensure(h->small, inblock_gs_scratch_doubles(b) * sizeof(double) + 64));
  BCHDAV_TRY(h->ensure_aux(256));
  HCUDA(cudaStreamSynchronize(st));   // earlier copies from host_aux are complete
  double* norm0_d = h->norm0.as<double>();
  double* fin_d = norm0_d + 64;
  int* dep_d = reinterpret_cast<int*>(norm0_d + 128);
  double* hp = h->host_aux;

  auto col_norms = [&](double* out_host) -> bchdav_status {
    // >= 16 rows per thread, within the partial-sum buffer
    const int nc = (int)std::min<size_t>(std::min(4 * kSMs, ceil_div(n, 256 / b * 16)),
                                         part_doubles / b);
    HCUDA(launch_col_sumsq_partial(st, n, X, ldx, b, h->part.as<double>(), nc));
    HCUDA(launch_reduce_partials(st, h->part.as<double>(), nc, b, h->G.as<double>(), 1.0));
    HCUDA(cudaMemcpyAsync(hp, h->G.as<double>(), b * sizeof(double), cudaMemcpyDeviceToHost, st));
    HCUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < b; ++j) out_host[j] = std::sqrt(hp[j]);
    return BCHDAV_OK;
  };

  std::vector<double> norm0(b);
  BCHDAV_TRY(col_norms(norm0.data()));
  *n_rep = 0;
  // tensor-core path: slices of V (by columns for V^T X, by rows for X -= V C) are made once
  // and serve both passes and every retry; X is sliced by columns for each Gram product
  if (vt_valid) *vt_valid = 0;
  const bool tc = (dense_path == 0 || dense_path == 2) && ozaki_nn_supported(std::max(k, 1));
  if (tc && dense_path == 0) BCHDAV_TRY(h->ensure(h->tc_err, sizeof(int)));
  const OzLayout L = oz_layout(n, std::max(k, cap_cols));
  const int Np = L.Np, capV = L.capV, capX = oz_pad_cols(b);
  const int Kp = oz_pad_k(std::max(k, 1));
  int *Evt = nullptr, *Evr = nullptr, *Ext = nullptr;
  if (tc) {
    BCHDAV_TRY(h->ensure(h->oz_vt, L.vt_planes + (size_t)oz_chunks(Np) * capV * sizeof(int) + 256));
    BCHDAV_TRY(h->ensure(h->oz_vr, L.vr_planes + (size_t)n * sizeof(int) + 256));
    BCHDAV_TRY(h->ensure(h->oz_xt, oz_planes_bytes(capX, Np) +
                                       (size_t)oz_chunks(Np) * capX * sizeof(int) + 256));
    BCHDAV_TRY(h->ensure(h->oz_bw, oz_bwork_bytes(std::max(k, b), std::max(b, 64))));
    BCHDAV_TRY(h->ensure(h->oz_part, (size_t)4 * kSMs * std::max(k, b) * b * sizeof(double)));
    Evt = reinterpret_cast<int*>(h->oz_vt.as<char>() + L.vt_planes);
    Evr = reinterpret_cast<int*>(h->oz_vr.as<char>() + L.vr_planes);
    Ext = reinterpret_cast<int*>(h->oz_xt.as<char>() + oz_planes_bytes(capX, Np));
    if (k > 0) {
      HCUDA(oz_slice_cols_t(st, n, V, ldv, k, Np, capV, 0, h->oz_vt.p, Evt));
      HCUDA(oz_slice_rows(st, n, V, ldv, k, Kp, h->oz_vr.p, Evr));
      if (vt_valid) *vt_valid = k;
    }
  }
  double* Gd = h->G.as<double>();
  bool vr_reused = false;   // the V row planes' buffer holds X's row planes (tensor-core CholQR)
  for (int attempt = 0; attempt < b + 16; ++attempt) {
    if (k > 0) {
      if (tc && vr_reused) {
        HCUDA(oz_slice_rows(st, n, V, ldv, k, Kp, h->oz_vr.p, Evr));
        vr_reused = false;
      }
      for (int pass = 0; pass < 2; ++pass) {
        if (tc) {
          // the second pass float64-accurate; the first from pass1_slices (8 on the float64 path:
          // a truncated first pass loosened its orthogonality on graphs with hub rows)
          HCUDA(oz_slice_cols_t(st, n, X, ldx, b, Np, capX, 0, h->oz_xt.p, Ext));
          HCUDA(gram_planes(h, dense_path, Np, h->oz_vt.p, Evt, capV, 0, k, h->oz_xt.p, Ext, capX,
                            b, Gd, pass == 0 ? pass1_slices : 8));
          if (dense_path == 0)
            HCUDA(oz_nn_from_planes_tc(st, n, k, Kp, h->oz_vr.p, Evr, Gd, b, b, X, ldx, true,
                                       h->oz_bw.p, 8, h->tc_err.as<int>()));
          else
            HCUDA(oz_nn_from_planes(st, n, k, Kp, h->oz_vr.p, Evr, Gd, b, b, X, ldx, true,
                                    h->oz_bw.p));
        } else {
          HCUDA(launch_gemm_tn_partial(st, n, V, ldv, k, X, ldx, b, h->part.as<double>(), chunks));
          HCUDA(launch_reduce_partials(st, h->part.as<double>(), chunks, k * b, Gd, 1.0));
          HCUDA(launch_gemm_nn_sub(st, n, V, ldv, k, Gd, b, b, X, ldx));
        }
      }
    }
    if (tc && b >= 2) {
      // inside the block: CholQR2 (X = Q R with G = X^T X = R^T R, twice).  R_jj is the norm
      // column j keeps after the earlier columns are projected out, i.e. the Gram-Schmidt
      // norm, so the dependence test is the same; whenever a pivot is small (or the test
      // fails) the exact column-by-column kernel below takes over.
      double* Rinv = Gd + g_words;
      int* flag = reinterpret_cast<int*>(Gd + g_words + 64 * 64);
      for (int j = 0; j < b; ++j) hp[j] = norm0[j];
      HCUDA(cudaMemcpyAsync(norm0_d, hp, b * sizeof(double), cudaMemcpyHostToDevice, st));
      bool ok = true;
      for (int pass = 0; pass < 2 && ok; ++pass) {
        // G = X^T X and X <- X R^{-1}: float64-accurate slice products on the tensor cores
        // (path 0; X's row planes go to the V row planes' buffer, free once both projections
        // are done), plain float64 otherwise
        if (dense_path == 0) {
          HCUDA(oz_slice_cols_t(st, n, X, ldx, b, Np, capX, 0, h->oz_xt.p, Ext));
          HCUDA(gram_planes(h, dense_path, Np, h->oz_xt.p, Ext, capX, 0, b, h->oz_xt.p, Ext, capX,
                            b, Gd));
        } else {
          HCUDA(launch_gemm_tn_partial(st, n, X, ldx, b, X, ldx, b, h->part.as<double>(), chunks));
          HCUDA(launch_reduce_partials(st, h->part.as<double>(), chunks, b * b, Gd, 1.0));
        }
        // the tensor-core product X R^{-1} slices the rows of X, each to one exponent: its
        // columns are first brought to comparable norms (exact powers of two, D), and
        // X R^{-1} = (X D) R'^{-1} with R' the Cholesky factor of D G D
        double* dscale = dense_path == 0 ? Gd + g_words + 64 * 64 + 8 : nullptr;
        HCUDA(launch_chol_inv(st, b, Gd, pass == 0 ? norm0_d : nullptr, pass == 0 ? 1e-4 : 0.5,
                              tau_dep, Rinv, flag, dscale));
        HCUDA(cudaMemcpyAsync(hp + 64, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        HCUDA(cudaStreamSynchronize(st));
        if (reinterpret_cast<int*>(hp + 64)[0] != 0) {
          ok = false;
          break;
        }
        if (dense_path == 0) {
          HCUDA(oz_slice_rows(st, n, X, ldx, b, oz_pad_k(b), h->oz_vr.p, Evr, dscale));
          vr_reused = true;
          HCUDA(oz_nn_from_planes_tc(st, n, b, oz_pad_k(b), h->oz_vr.p, Evr, Rinv, b, b, X, ldx,
                                     false, h->oz_bw.p, 8, h->tc_err.as<int>()));
        } else {
          HCUDA(launch_gemm_tri_inplace(st, n, X, ldx, b, Rinv, b));
        }
      }
      if (ok) return BCHDAV_OK;
      // a failed first pass left X untouched; a failed second pass (never expected after a
      // successful first) leaves X orthogonal enough for the exact kernel to finish
    }
    for (int j = 0; j < b; ++j) hp[j] = norm0[j];
    reinterpret_cast<int*>(hp + 64)[0] = -1;
    HCUDA(cudaMemcpyAsync(norm0_d, hp, b * sizeof(double), cudaMemcpyHostToDevice, st));
    HCUDA(cudaMemcpyAsync(dep_d, hp + 64, sizeof(int), cudaMemcpyHostToDevice, st));
    HCUDA(launch_inblock_gs(st, n, X, ldx, b, 0, norm0_d, tau_dep, h->small.as<double>(), dep_d,
                            fin_d, h->coop_grid_cap));
    HCUDA(cudaMemcpyAsync(hp + 64, dep_d, sizeof(int), cudaMemcpyDeviceToHost, st));
    HCUDA(cudaStreamSynchronize(st));
    const int dep = reinterpret_cast<int*>(hp + 64)[0];
    if (dep < 0) return BCHDAV_OK;
    HCUDA(launch_fill_random_col(st, n, X, ldx, dep, seed, kStreamReplace,
                                 (uint32_t)(*rep_counter)));
    ++(*rep_counter);
    ++(*n_rep);
    std::vector<double> nn(b);
    BCHDAV_TRY(col_norms(nn.data()));
    for (int j = 0; j < dep; ++j) norm0[j] = 1.0;
    norm0[dep] = nn[dep];
  }
  h->set_error(BCHDAV_ERR_NONFINITE, "orthonormalisation: replacement vectors keep failing");
  return BCHDAV_ERR_NONFINITE;
}

double median_of(std::vector<double> v) {
  std::sort(v.begin(), v.end());
  size_t n = v.size();
  if (n % 2 == 1) return v[n / 2];
  return 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

}  // namespace

// Long-row schedule (declared in handle.cuh).  Rebuilt on every call: it costs one pass over
// rowptr and one host synchronisation.
bchdav_status prepare_long_rows(bchdav_handle h, const bchdav_csr* A, size_t width_bytes) {
  cudaStream_t st = h->stream;
  const int n = A->n;
  h->lg = bchdav::SpmmLong();
  const long long cap = spmm_long_seg_cap(A->nnz);
  BCHDAV_TRY(h->ensure(h->lg_cnt, (size_t)n * sizeof(int)));
  BCHDAV_TRY(h->ensure(h->lg_off, (size_t)(n + 1) * sizeof(long long)));
  BCHDAV_TRY(h->ensure(h->lg_tiles, (size_t)scan_tile_count(n) * sizeof(long long) + 64));
  BCHDAV_TRY(h->ensure(h->lg_row, (size_t)cap * sizeof(int)));
  long long total = 0, n_seg = 0;
  HCUDA(build_spmm_long(st, n, A->rowptr, h->lg_cnt.as<int>(), h->lg_off.as<long long>(),
                        h->lg_tiles.as<long long>(), h->lg_row.as<int>(), cap, &total, &n_seg));
  if (n_seg > 0) {
    BCHDAV_TRY(h->ensure(h->lg_pseg, (size_t)n_seg * width_bytes));
    h->lg.n_seg = n_seg;
    h->lg.seg_off = h->lg_off.as<long long>();
    h->lg.seg_row = h->lg_row.as<int>();
    h->lg.pseg = h->lg_pseg.p;
  }
  return BCHDAV_OK;
}

namespace bchdav {
// Message returned by bchdav_last_error(NULL) for entry points without a handle.
void set_global_error(const char* msg) { g_create_error = msg; }
}  // namespace bchdav

// =====================================================================
extern "C" {

const char* bchdav_status_string(bchdav_status s) {
  switch (s) {
    case BCHDAV_OK: return "ok";
    case BCHDAV_NOT_CONVERGED: return "not converged (itmax reached)";
    case BCHDAV_ERR_ARG: return "invalid argument";
    case BCHDAV_ERR_CSR: return "invalid CSR matrix";
    case BCHDAV_ERR_OOM: return "out of device memory";
    case BCHDAV_ERR_CUDA: return "CUDA error";
    case BCHDAV_ERR_NONFINITE: return "non-finite value in the iteration";
    case BCHDAV_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

bchdav_status bchdav_create(bchdav_handle* out, void* stream) {
  if (!out) return BCHDAV_ERR_ARG;
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_create_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return BCHDAV_ERR_CUDA;
  }
  bchdav_handle h = new bchdav_handle_s();
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->device = dev;
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  *out = h;
  return BCHDAV_OK;
}

bchdav_status bchdav_destroy(bchdav_handle h) {
  if (!h) return BCHDAV_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  h->release_all();
  delete h;
  return BCHDAV_OK;
}

bchdav_status bchdav_set_memory_limit(bchdav_handle h, uint64_t bytes) {
  if (!h) return BCHDAV_ERR_ARG;
  h->mem_limit = (size_t)bytes;
  return BCHDAV_OK;
}

uint64_t bchdav_workspace_bytes(bchdav_handle h) { return h ? (uint64_t)h->held_bytes() : 0; }

bchdav_status bchdav_set_stream(bchdav_handle h, void* stream) {
  if (!h) return BCHDAV_ERR_ARG;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  return BCHDAV_OK;
}

const char* bchdav_last_error(bchdav_handle h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

int32_t bchdav_history(bchdav_handle h, bchdav_iter_record* out, int32_t max_records) {
  if (!h) return 0;
  int32_t n = (int32_t)h->history.size();
  if (out && max_records > 0) {
    int32_t c = std::min(n, max_records);
    std::memcpy(out, h->history.data(), c * sizeof(bchdav_iter_record));
  }
  return n;
}

bchdav_status bchdav_spmm(bchdav_handle h, const bchdav_csr* A, const double* X, int32_t ldx,
                          int32_t b, double* Y, int32_t ldy) {
  if (!h) return BCHDAV_ERR_ARG;
  BCHDAV_TRY(check_csr_args(h, A));
  if (b < 1 || ldx < b || ldy < b || !X || !Y) {
    h->set_error(BCHDAV_ERR_ARG, "spmm: bad block arguments");
    return BCHDAV_ERR_ARG;
  }
  BCHDAV_TRY(prepare_long_rows(h, A, (size_t)b * sizeof(double)));
  HCUDA(launch_spmm_axpby<double>(h->stream, A->n, A->rowptr, A->colidx, A->val, X, ldx, b, Y, ldy,
                                  nullptr, 0, 1.0, 0.0, 0.0, nullptr, 0, nullptr, h->long_rows()));
  return BCHDAV_OK;
}

bchdav_status bchdav_spmm_dd(bchdav_handle h, const bchdav_csr* A, const double* X, int32_t ldx,
                             int32_t b, double* Y, int32_t ldy) {
  if (!h) return BCHDAV_ERR_ARG;
  BCHDAV_TRY(check_csr_args(h, A));
  if (b < 1 || ldx < b || ldy < b || !X || !Y || X == Y || !A->val_f32) {
    h->set_error(BCHDAV_ERR_ARG, "spmm_dd: bad arguments (A->val_f32 required, X != Y)");
    return BCHDAV_ERR_ARG;
  }
  BCHDAV_TRY(prepare_long_rows(h, A, (size_t)b * sizeof(double)));
  if (!spmm_dd_supported(b, h->long_rows())) {
    h->set_error(BCHDAV_ERR_ARG,
                 "spmm_dd: b must be a multiple of 4 (<= 128) and no row may need segments");
    return BCHDAV_ERR_ARG;
  }
  BCHDAV_TRY(h->ensure(h->vallo, (size_t)A->nnz * sizeof(float)));
  BCHDAV_TRY(h->ensure(h->ddx, spmm_dd_scratch_floats(A->n, b) * sizeof(float)));
  HCUDA(launch_split_dd_vec(h->stream, A->nnz, A->val, h->vallo.as<float>()));
  HCUDA(launch_spmm_dd(h->stream, A->n, A->rowptr, A->colidx, A->val_f32, h->vallo.as<float>(), X,
                       ldx, b, Y, ldy, 1.0, nullptr, 0, nullptr, h->ddx.as<float>()));
  return BCHDAV_OK;
}

bchdav_status bchdav_filter(bchdav_handle h, const bchdav_csr* A, const double* X, int32_t ldx,
                            int32_t b, int32_t m, double a, double upb, double a0,
                            int32_t precision, double* Y, int32_t ldy) {
  if (!h) return BCHDAV_ERR_ARG;
  BCHDAV_TRY(check_csr_args(h, A));
  if (b < 1 || m < 1 || ldx < b || ldy < b || !X || !Y || X == Y || !(upb > a) || !(a0 < a)) {
    h->set_error(BCHDAV_ERR_ARG, "filter: bad arguments (need a0 < a < upb, m >= 1)");
    return BCHDAV_ERR_ARG;
  }
  const float* v32 = A->val_f32;
  if (precision == BCHDAV_PREC_MIXED && !v32) {
    BCHDAV_TRY(h->ensure(h->val32, (size_t)A->nnz * sizeof(float)));
    HCUDA(launch_f64_to_f32_vec(h->stream, A->nnz, A->val, h->val32.as<float>()));
    v32 = h->val32.as<float>();
  }
  BCHDAV_TRY(prepare_long_rows(h, A, (size_t)b * sizeof(double)));
  return run_filter(h, A, v32, X, ldx, b, m, a, upb, a0, precision, Y, ldy, nullptr);
}

bchdav_status bchdav_orthonormalize(bchdav_handle h, int32_t n, const double* V, int32_t ldv,
                                    int32_t k, double* X, int32_t ldx, int32_t b, uint64_t seed,
                                    double tau_dep, int64_t* rep_counter, int32_t* n_replaced) {
  if (!h) return BCHDAV_ERR_ARG;
  if (n < 1 || b < 1 || b > 64 || k < 0 || k + b > n || ldx < b || (k > 0 && (!V || ldv < k)) ||
      !X || !rep_counter) {
    h->set_error(BCHDAV_ERR_ARG, "orthonormalize: bad arguments");
    return BCHDAV_ERR_ARG;
  }
  if (k > 768) {
    h->set_error(BCHDAV_ERR_ARG, "orthonormalize: basis wider than supported (768)");
    return BCHDAV_ERR_ARG;
  }
  int nr = 0;
  BCHDAV_TRY(h->ensure(h->tc_err, sizeof(int)));
  HCUDA(cudaMemsetAsync(h->tc_err.p, 0, sizeof(int), h->stream));
  bchdav_status s = run_orth(h, n, V, ldv, k, X, ldx, b, seed, tau_dep, rep_counter, &nr);
  if (n_replaced) *n_replaced = nr;
  if (s != BCHDAV_OK) return s;
  int flag = 0;
  HCUDA(cudaMemcpyAsync(&flag, h->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HCUDA(cudaStreamSynchronize(h->stream));
  if (flag) {
    h->set_error(BCHDAV_ERR_TIMEOUT, "orthonormalize: a tensor-core wait expired");
    return BCHDAV_ERR_TIMEOUT;
  }
  return s;
}

bchdav_status bchdav_gram(bchdav_handle h, int32_t n, const double* A, int32_t lda, int32_t ka,
                          const double* B, int32_t ldb, int32_t kb, double* out,
                          int32_t dense_path) {
  if (!h) return BCHDAV_ERR_ARG;
  if (n < 1 || ka < 1 || kb < 1 || lda < ka || ldb < kb || !A || !B || !out ||
      dense_path < 0 || dense_path > 2 || (size_t)ka * kb > 16 * 1024 * 1024) {
    h->set_error(BCHDAV_ERR_ARG, "gram: bad arguments");
    return BCHDAV_ERR_ARG;
  }
  if (dense_path != 1) {
    BCHDAV_TRY(h->ensure(h->oz, ozaki_tn_work_bytes(n, ka, kb)));
    int* err = nullptr;
    if (dense_path == 0) {
      BCHDAV_TRY(h->ensure(h->tc_err, sizeof(int)));
      HCUDA(cudaMemsetAsync(h->tc_err.p, 0, sizeof(int), h->stream));
      err = h->tc_err.as<int>();
    }
    HCUDA(launch_ozaki_tn(h->stream, n, A, lda, ka, B, ldb, kb, out, h->oz.p, err));
    if (err) {
      int flag = 0;
      HCUDA(cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      HCUDA(cudaStreamSynchronize(h->stream));
      if (flag) {
        h->set_error(BCHDAV_ERR_TIMEOUT, "gram: a tensor-core wait expired");
        return BCHDAV_ERR_TIMEOUT;
      }
    }
  } else {
    const int chunks = gemm_tn_chunks(n);
    BCHDAV_TRY(h->ensure(h->part, (size_t)chunks * ka * kb * sizeof(double)));
    HCUDA(launch_gemm_tn_partial(h->stream, n, A, lda, ka, B, ldb, kb, h->part.as<double>(), chunks));
    HCUDA(launch_reduce_partials(h->stream, h->part.as<double>(), chunks, ka * kb, out, 1.0));
  }
  return BCHDAV_OK;
}

bchdav_status bchdav_rotate(bchdav_handle h, int32_t n, double* V, int32_t ldv, int32_t k,
                            const double* Y, int32_t ld_y, int32_t nb, int32_t dense_path) {
  if (!h) return BCHDAV_ERR_ARG;
  if (n < 1 || k < 1 || nb < 1 || nb > k || ldv < k || ld_y < nb || !V || !Y ||
      dense_path < 0 || dense_path > 2) {
    h->set_error(BCHDAV_ERR_ARG, "rotate: bad arguments");
    return BCHDAV_ERR_ARG;
  }
  if (dense_path == 0 && ozaki_nn_supported(k)) {
    // tcgen05 slice product from V's row planes (in place: the planes hold all of V)
    const int Kp = oz_pad_k(k);
    BCHDAV_TRY(h->ensure(h->oz, oz_planes_bytes(n, Kp) + (size_t)n * sizeof(int) + 256));
    BCHDAV_TRY(h->ensure(h->oz_bw, oz_bwork_bytes(k, nb)));
    BCHDAV_TRY(h->ensure(h->tc_err, sizeof(int)));
    int* E = reinterpret_cast<int*>(h->oz.as<char>() + oz_planes_bytes(n, Kp));
    HCUDA(cudaMemsetAsync(h->tc_err.p, 0, sizeof(int), h->stream));
    HCUDA(oz_slice_rows(h->stream, n, V, ldv, k, Kp, h->oz.p, E));
    HCUDA(oz_nn_from_planes_tc(h->stream, n, k, Kp, h->oz.p, E, Y, ld_y, nb, V, ldv, false,
                               h->oz_bw.p, 8, h->tc_err.as<int>()));
    int flag = 0;
    HCUDA(cudaMemcpyAsync(&flag, h->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    HCUDA(cudaStreamSynchronize(h->stream));
    if (flag) {
      h->set_error(BCHDAV_ERR_TIMEOUT, "rotate: a tensor-core wait expired");
      return BCHDAV_ERR_TIMEOUT;
    }
  } else if (dense_path == 2 && ozaki_nn_supported(k)) {
    BCHDAV_TRY(h->ensure(h->oz, ozaki_nn_work_bytes(n, k, nb)));
    HCUDA(launch_ozaki_nn(h->stream, n, V, ldv, k, Y, ld_y, nb, V, ldv, false, h->oz.p));
  } else {
    HCUDA(launch_gemm_nn_inplace(h->stream, n, V, ldv, k, Y, ld_y, nb));
  }
  return BCHDAV_OK;
}

bchdav_status bchdav_eigh(bchdav_handle h, int32_t n, const double* H, int32_t ld_h, double* D,
                          double* Y, int32_t ld_y) {
  if (!h) return BCHDAV_ERR_ARG;
  if (n < 1 || n > 1024 || ld_h < n || ld_y < n || !H || !D || !Y) {
    h->set_error(BCHDAV_ERR_ARG, n > 1024 ? "eigh: n is limited to 1024"
                                          : "eigh: bad arguments");
    return BCHDAV_ERR_ARG;
  }
  const size_t wd = std::max(eigh_work_doubles(n), eigh_fast_work_doubles(n));
  BCHDAV_TRY(h->ensure(h->eigw, wd * sizeof(double) + 64));
  int* status_d = reinterpret_cast<int*>(h->eigw.as<char>() + wd * sizeof(double));
  const bool aux = h->ensure_aux_stream();
  HCUDA(launch_eigh_fast(h->stream, n, H, ld_h, D, Y, ld_y, h->eigw.as<double>(), status_d,
                         h->coop_grid_cap, aux ? h->aux_stream : nullptr,
                         aux ? h->aux_ev[0] : nullptr, aux ? h->aux_ev[1] : nullptr));
  int st = 0;
  HCUDA(cudaMemcpyAsync(&st, status_d, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HCUDA(cudaStreamSynchronize(h->stream));
  if (st == 2) {
    h->set_error(BCHDAV_ERR_TIMEOUT, "eigh: a grid barrier of the eigensolver gave up waiting");
    return BCHDAV_ERR_TIMEOUT;
  }
  if (st != 0) {
    h->set_error(BCHDAV_ERR_NONFINITE, "eigh: the iteration did not converge");
    return BCHDAV_ERR_NONFINITE;
  }
  return BCHDAV_OK;
}

// ---------------------------------------------------------------------
bchdav_status bchdav_solve(bchdav_handle h, const bchdav_csr* A, int32_t k, int32_t b, int32_t m,
                           int32_t act_max_in, double tol, const bchdav_opts* opts_in,
                           double* evals, double* evecs, bchdav_info* info) {
  if (!h) return BCHDAV_ERR_ARG;
  BCHDAV_TRY(check_csr_args(h, A));
  bchdav_opts opts;
  std::memset(&opts, 0, sizeof(opts));
  if (opts_in) opts = *opts_in;
  const int N = A->n;
  const int act_max = act_max_in > 0 ? act_max_in : std::max(5 * b, 30);
  int dim_max = opts.dim_max > 0 ? opts.dim_max : std::min(std::max(act_max + 2 * b, k + 30), N);
  const int itmax = opts.itmax > 0 ? opts.itmax : 1000;
  const int prec = opts.precision;
  if (k < 1 || k > N || b < 1 || b > 64 || m < 1 || act_max < 2 * b || act_max > N ||
      !(tol > 0) || !evals || !evecs || (prec != BCHDAV_PREC_FP64 && prec != BCHDAV_PREC_MIXED) ||
      (opts.k_init > 0 && (!opts.v_init || opts.ld_v_init < opts.k_init)) ||
      opts.dense_path < 0 || opts.dense_path > 2 || opts.bounds < BCHDAV_BOUNDS_NORMALIZED ||
      opts.bounds > BCHDAV_BOUNDS_LANCZOS ||
      (opts.bounds == BCHDAV_BOUNDS_GIVEN &&
       !(std::isfinite(opts.lowb) && std::isfinite(opts.upperb) && opts.lowb < opts.upperb)) ||
      (opts.bounds == BCHDAV_BOUNDS_LANCZOS &&
       (opts.lanczos_steps < 0 || opts.lanczos_steps > 64 || opts.lanczos_steps > N))) {
    h->set_error(BCHDAV_ERR_ARG, "solve: invalid k, b, m, act_max, tol or options");
    return BCHDAV_ERR_ARG;
  }
  const int ncols = std::max(dim_max, k + 2 * b);
  if (ncols > N || dim_max < act_max) {
    h->set_error(BCHDAV_ERR_ARG, "solve: subspace (dim_max, k + 2b) larger than N or below act_max");
    return BCHDAV_ERR_ARG;
  }
  if (act_max > 768 || ncols > 768) {
    h->set_error(BCHDAV_ERR_ARG, "solve: act_max and dim_max are limited to 768");
    return BCHDAV_ERR_ARG;
  }
  const int k_ri = std::max(act_max / 2, act_max - 3 * b);
  cudaStream_t st = h->stream;
  const double tau_dep = prec == BCHDAV_PREC_MIXED ? kTauDepMixed : kTauDepF64;

  // A caller's initial block must be finite: one NaN would spread through the filter into
  // every later vector.  Checked once here (one pass over N x k_init) so that such an input
  // fails at once with BCHDAV_ERR_NONFINITE instead of after a wasted iteration.
  if (opts.k_init > 0) {
    BCHDAV_TRY(h->ensure(h->vchk, sizeof(int)));
    BCHDAV_TRY(h->ensure_pinned(1024));
    HCUDA(cudaMemsetAsync(h->vchk.p, 0, sizeof(int), st));
    HCUDA(launch_check_finite(st, N, opts.k_init, opts.v_init, opts.ld_v_init, h->vchk.as<int>()));
    int* flag_h = reinterpret_cast<int*>(h->host_pinned);
    HCUDA(cudaMemcpyAsync(flag_h, h->vchk.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HCUDA(cudaStreamSynchronize(st));
    if (*flag_h != 0) {
      h->set_error(BCHDAV_ERR_NONFINITE, "solve: v_init holds a non-finite value");
      return BCHDAV_ERR_NONFINITE;
    }
  }

  // ---- workspace
  // W = A V (Algorithm 2, Steps 7, 11, 14): only its newest k_b columns are ever read (Step 8
  // builds the new columns of H from them; Step 12 recomputes A V itself), so the driver keeps
  // just those columns and skips rotating and shifting the older ones, whose values no step
  // reads.  Every output is unchanged.
  const int ldv = round_up(ncols, 2), ldb = round_up(b, 2);
  BCHDAV_TRY(h->ensure(h->V, (size_t)N * ldv * sizeof(double)));
  BCHDAV_TRY(h->ensure(h->W, (size_t)N * ldb * sizeof(double)));
  BCHDAV_TRY(h->ensure(h->Vtmp, (size_t)N * ldb * sizeof(double)));
  BCHDAV_TRY(h->ensure(h->Xo, (size_t)N * ldb * sizeof(double)));
  BCHDAV_TRY(h->ensure(h->R, (size_t)N * ldb * sizeof(double)));
  BCHDAV_TRY(h->ensure(h->H, (size_t)act_max * act_max * sizeof(double)));
  BCHDAV_TRY(h->ensure(h->Y, (size_t)act_max * act_max * sizeof(double)));
  BCHDAV_TRY(h->ensure(h->D, (size_t)(act_max + 256 + ncols + 64 + 128) * sizeof(double)));
  const size_t eig_wd = std::max(eigh_work_doubles(act_max), eigh_fast_work_doubles(act_max));
  BCHDAV_TRY(h->ensure(h->eigw, eig_wd * sizeof(double) + 64));
  const int chunks = gemm_tn_chunks(N);
  const int rparts = spmm_resid_max_parts(N, b);
  BCHDAV_TRY(h->ensure(h->part, std::max((size_t)chunks * ncols * b,
                                          (size_t)std::max(rparts, chunks) * 2 * 128) *
                                    sizeof(double)));
  BCHDAV_TRY(h->ensure(h->G, (size_t)std::max(ncols * b, 64) * sizeof(double)));
  BCHDAV_TRY(h->ensure_pinned((size_t)std::max(4 * act_max + 4 * ncols, 1024)));
  BCHDAV_TRY(h->ensure_aux((size_t)(m + 1) * 64 + 256));
  // tensor-core products: V's column planes (Steps 6, 8) and row planes (Steps 6, 11) sized for
  // the whole subspace, X / W column planes, the split-B work and the split-reduction partials
  const OzLayout OL = oz_layout(N, ncols);
  // Step 11 rotation: the float64 path keeps all 8 digit slices (48-bit operands); the mixed
  // path takes 6 (36-bit operands, ~2e-11 relative per rotation), far below its float32
  // filter's rounding and the 1e-8 residual target.  Step 8's H stays at 8 slices: its Ritz
  // values decide convergence, and a hub row's chunk costs the other rows bits there.
  const int slices_rr = prec == BCHDAV_PREC_MIXED ? 6 : 8;
  BCHDAV_TRY(h->ensure(h->tc_err, sizeof(int)));
  HCUDA(cudaMemsetAsync(h->tc_err.p, 0, sizeof(int), st));
  if (opts.dense_path != 1) {
    BCHDAV_TRY(h->ensure(h->oz_vt, OL.vt_planes + (size_t)oz_chunks(OL.Np) * OL.capV * sizeof(int) +
                                       256));
    BCHDAV_TRY(h->ensure(h->oz_vr, OL.vr_planes + (size_t)N * sizeof(int) + 256));
    BCHDAV_TRY(h->ensure(h->oz_xt, oz_planes_bytes(oz_pad_cols(b), OL.Np) +
                                       (size_t)oz_chunks(OL.Np) * oz_pad_cols(b) * sizeof(int) + 256));
    BCHDAV_TRY(h->ensure(h->oz_bw, oz_bwork_bytes(std::max(ncols, act_max), std::max(act_max, 64))));
    BCHDAV_TRY(h->ensure(h->oz_part, (size_t)4 * kSMs * ncols * b * sizeof(double)));
  }
  const float* val32 = A->val_f32;
  if (prec == BCHDAV_PREC_MIXED && !val32) {
    BCHDAV_TRY(h->ensure(h->val32, (size_t)A->nnz * sizeof(float)));
    HCUDA(launch_f64_to_f32_vec(st, A->nnz, A->val, h->val32.as<float>()));
    val32 = h->val32.as<float>();
  }
  BCHDAV_TRY(prepare_long_rows(h, A, (size_t)std::max(2 * b, 64) * sizeof(double)));
  // mixed path: Steps 7 and 12 as double-float products (A's values as float hi + lo, hi the
  // float32 copy of the filter), where the block width allows and no row is segmented
  const bool dd = prec == BCHDAV_PREC_MIXED && spmm_dd_supported(b, h->long_rows());
  const float* val_lo = nullptr;
  float* dd_scr = nullptr;
  if (dd) {
    BCHDAV_TRY(h->ensure(h->vallo, (size_t)A->nnz * sizeof(float)));
    BCHDAV_TRY(h->ensure(h->ddx, spmm_dd_scratch_floats(N, b) * sizeof(float)));
    HCUDA(launch_split_dd_vec(st, A->nnz, A->val, h->vallo.as<float>()));
    val_lo = h->vallo.as<float>();
    dd_scr = h->ddx.as<float>();
  }
  double* V = h->V.as<double>();
  double* W = h->W.as<double>();
  double* Vtmp = h->Vtmp.as<double>();
  double* Xo = h->Xo.as<double>();
  double* Hm = h->H.as<double>();
  double* Ym = h->Y.as<double>();
  double* Dd = h->D.as<double>();            // act_max Ritz values
  double* dsel = Dd + act_max;               // device staging for small vectors (256)
  int* perm_d = reinterpret_cast<int*>(dsel + 256);   // ncols column indices
  double* negd = Dd + act_max + 256 + ncols + 64;      // 128: -d of the residual epilogue
  int* eig_status = reinterpret_cast<int*>(h->eigw.as<char>() + eig_wd * sizeof(double));
  double* hp = h->host_pinned;
  h->history.clear();

  Timer tm_total, tm_filter, tm_orth, tm_spmm, tm_h, tm_eig, tm_rot, tm_res, tm_res2;
  Timer* timers[] = {&tm_total, &tm_filter, &tm_orth, &tm_spmm, &tm_h,
                     &tm_eig,   &tm_rot,    &tm_res,  &tm_res2};
  for (Timer* t : timers) t->init();
  struct Cleanup {
    Timer** t;
    int n;
    ~Cleanup() {
      for (int i = 0; i < n; ++i) t[i]->destroy();
    }
  } cleanup{timers, 8};
  auto collect = [&]() {
    for (Timer* t : timers)
      if (t != &tm_total) t->collect();
  };
  double filter_bytes = 0.0;
  const unsigned long long launches0 = __atomic_load_n(&bchdav::g_launches, __ATOMIC_RELAXED);
  tm_total.start(st);

  // ---- Step 1: bounds (analytic for Eq. (1), given, or by k-step Lanczos)
  double lowb = 0.0, upperb = 2.0;
  if (opts.bounds == BCHDAV_BOUNDS_GIVEN) {
    lowb = opts.lowb;
    upperb = opts.upperb;
  } else if (opts.bounds == BCHDAV_BOUNDS_LANCZOS) {
    const int steps = opts.lanczos_steps > 0 ? opts.lanczos_steps : std::min(20, N);
    BCHDAV_TRY(bchdav::lanczos_bounds(h, A, steps, opts.seed, &lowb, &upperb, nullptr, nullptr,
                                      nullptr));
    if (!(upperb > lowb)) {
      h->set_error(BCHDAV_ERR_ARG, "solve: the Lanczos estimate gives lowb >= upperb "
                                   "(a multiple of the identity?)");
      return BCHDAV_ERR_ARG;
    }
  }
  double low_nwb = lowb + (upperb - lowb) * (double)k / (double)N;

  // ---- Step 2: first filter input
  const int k_init = opts.k_init > 0 ? opts.k_init : 0;
  const int n_first = std::min(b, k_init);
  if (n_first > 0) HCUDA(launch_copy_block(st, N, n_first, opts.v_init, opts.ld_v_init, Vtmp, ldb));
  uint32_t fill_counter = 0;
  for (int j = n_first; j < b; ++j)
    HCUDA(launch_fill_random_col(st, N, Vtmp, ldb, j, opts.seed, kStreamFill, fill_counter++));
  int k_i = n_first;

  // ---- Step 3
  int k_c = 0, k_sub = 0, k_act = 0;
  std::vector<double> eval_locked;
  int64_t rep_counter = 0;
  int n_rep_total = 0, n_spmm = 0, it = 0;
  bool converged = false;
  std::vector<double> Dh(act_max);
  // mixed path: per filter-input column, the tested column of Step 12 whose residual it
  // filters (-1: plain column) and its Ritz value
  std::vector<int> mix_src(b, -1);
  std::vector<double> mix_theta(b, NAN);
  const int ldr = round_up(2 * b, 2);
  BCHDAV_TRY(h->ensure(h->Rres, (size_t)N * ldr * sizeof(double)));   // Step 12 residual block

  while (it < itmax) {
    ++it;
    // Step 5: Chebyshev filter
    tm_filter.start(st);
    if (prec == BCHDAV_PREC_MIXED) {
      BCHDAV_TRY(run_filter_mixed(h, A, val32, Vtmp, ldb, h->Rres.as<double>(), ldr, mix_src.data(),
                                  mix_theta.data(), b, m, low_nwb, upperb, lowb, Xo, ldb,
                                  &filter_bytes));
    } else {
      BCHDAV_TRY(run_filter(h, A, val32, Vtmp, ldb, b, m, low_nwb, upperb, lowb, prec, Xo, ldb,
                            &filter_bytes));
    }
    tm_filter.stop(st);
    n_spmm += m;
    // Step 6: orthonormalise against V(:, 1:k_sub)
    tm_orth.start(st);
    int nrep = 0;
    const int k_orth = k_sub;
    int vt_valid = 0;
    BCHDAV_TRY(run_orth(h, N, V, ldv, k_sub, Xo, ldb, b, opts.seed, tau_dep, &rep_counter, &nrep,
                        opts.dense_path, ncols, &vt_valid,
                        prec == BCHDAV_PREC_MIXED ? kMixedPass1Slices : 8));
    n_rep_total += nrep;
    HCUDA(launch_copy_block(st, N, b, Xo, ldb, V + k_sub, ldv));
    tm_orth.stop(st);
    // Step 7: W(:, k_act+1 : k_act+b) = A V_new
    tm_spmm.start(st);
    if (dd)
      HCUDA(launch_spmm_dd(st, N, A->rowptr, A->colidx, val32, val_lo, Xo, ldb, b, W, ldb, 1.0,
                           nullptr, 0, nullptr, dd_scr));
    else
      HCUDA(launch_spmm_axpby<double>(st, N, A->rowptr, A->colidx, A->val, Xo, ldb, b, W, ldb,
                                      nullptr, 0, 1.0, 0.0, 0.0, nullptr, 0, nullptr,
                                      h->long_rows()));
    tm_spmm.stop(st);
    ++n_spmm;
    k_act += b;
    k_sub += b;
    // Step 8: H(1:k_act, new) = V(:, k_c+1:k_sub)^T W_new, symmetrise
    tm_h.start(st);
    if (opts.dense_path != 1) {
      // V's column planes from Step 6 are still current for columns [0, vt_valid); slice the
      // rest of V(:, k_c+1:k_sub) (the new block) and W_new, then reduce over the N rows
      int* Evt = reinterpret_cast<int*>(h->oz_vt.as<char>() + OL.vt_planes);
      const int capX = oz_pad_cols(b);
      int* Ext = reinterpret_cast<int*>(h->oz_xt.as<char>() + oz_planes_bytes(capX, OL.Np));
      const int c_from = std::max(vt_valid, k_c);
      HCUDA(oz_slice_cols_t(st, N, V + c_from, ldv, k_sub - c_from, OL.Np, OL.capV, c_from,
                            h->oz_vt.p, Evt));
      HCUDA(oz_slice_cols_t(st, N, W, ldb, b, OL.Np, capX, 0, h->oz_xt.p, Ext));
      // float64-accurate on both paths: only the newest b columns of H are formed, the old
      // block is the diagonal of the previous Ritz values, so an early truncated product would
      // leave its error in diagonal entries that no later product refreshes
      HCUDA(gram_planes(h, opts.dense_path, OL.Np, h->oz_vt.p, Evt, OL.capV, k_c, k_act,
                        h->oz_xt.p, Ext, capX, b, h->G.as<double>()));
    } else {
      HCUDA(launch_gemm_tn_partial(st, N, V + k_c, ldv, k_act, W, ldb, b, h->part.as<double>(),
                                   chunks));
      HCUDA(launch_reduce_partials(st, h->part.as<double>(), chunks, k_act * b, h->G.as<double>(),
                                   1.0));
    }
    HCUDA(launch_h_update(st, Hm, act_max, h->G.as<double>(), k_act, b));
    tm_h.stop(st);
    // Step 9: H Y = Y D (ascending)
    tm_eig.start(st);
    {
      const bool aux = h->ensure_aux_stream();
      HCUDA(launch_eigh_fast(st, k_act, Hm, act_max, Dd, Ym, act_max, h->eigw.as<double>(),
                             eig_status, h->coop_grid_cap, aux ? h->aux_stream : nullptr,
                             aux ? h->aux_ev[0] : nullptr, aux ? h->aux_ev[1] : nullptr));
    }
    tm_eig.stop(st);
    HCUDA(cudaMemcpyAsync(hp, Dd, k_act * sizeof(double), cudaMemcpyDeviceToHost, st));
    HCUDA(cudaMemcpyAsync(hp + act_max, eig_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    const int k_old = k_act;
    // Step 10: inner restart
    if (k_act + b > act_max) {
      k_act = k_ri;
      k_sub = k_act + k_c;
    }
    // Step 11: rotation V(:, k_c+1 : k_c+k_act) = V(:, k_c+1 : k_c+k_old) Y(:, 1:k_act)
    tm_rot.start(st);
    if (opts.dense_path != 1 && ozaki_nn_supported(k_old)) {
      // the row planes of Step 6 are stale (V gained a block); re-slice V(:, k_c+1:k_c+k_old)
      // into the same buffer, then V is overwritten in place (the planes hold all of A)
      int* Evr = reinterpret_cast<int*>(h->oz_vr.as<char>() + OL.vr_planes);
      const int Kp = oz_pad_k(k_old);
      HCUDA(oz_slice_rows(st, N, V + k_c, ldv, k_old, Kp, h->oz_vr.p, Evr, nullptr,
                          opts.dense_path == 0 ? slices_rr : 8));
      if (opts.dense_path == 0)
        HCUDA(oz_nn_from_planes_tc(st, N, k_old, Kp, h->oz_vr.p, Evr, Ym, act_max, k_act, V + k_c,
                                   ldv, false, h->oz_bw.p, slices_rr, h->tc_err.as<int>()));
      else
        HCUDA(oz_nn_from_planes(st, N, k_old, Kp, h->oz_vr.p, Evr, Ym, act_max, k_act, V + k_c,
                                ldv, false, h->oz_bw.p, slices_rr));
    } else {
      HCUDA(launch_gemm_nn_inplace(st, N, V + k_c, ldv, k_old, Ym, act_max, k_act));
    }
    tm_rot.stop(st);
    // Step 12: residuals of the leading k_b Ritz pairs
    const int nt = std::min(b, k_act);
    const int nres = nt;
    tm_res.start(st);
    int nparts = 0;
    if (dd && nres % 4 == 0)
      HCUDA(launch_spmm_resid_dd(st, N, A->rowptr, A->colidx, val32, val_lo, V + k_c, ldv, nres,
                                 Dd, h->part.as<double>(), &nparts, h->Rres.as<double>(), ldr,
                                 negd, dd_scr));
    else
      HCUDA(launch_spmm_resid(st, N, A->rowptr, A->colidx, A->val, V + k_c, ldv, nres, Dd,
                              h->part.as<double>(), &nparts, h->Rres.as<double>(), ldr, negd,
                              h->long_rows()));
    HCUDA(launch_reduce_partials(st, h->part.as<double>(), nparts, 2 * nres, dsel, 1.0));
    HCUDA(cudaMemcpyAsync(hp + act_max + 1, dsel, 2 * nres * sizeof(double), cudaMemcpyDeviceToHost,
                          st));
    tm_res.stop(st);
    ++n_spmm;
    HCUDA(cudaStreamSynchronize(st));
    collect();
    if (reinterpret_cast<int*>(hp + act_max)[0] == 2) {
      h->set_error(BCHDAV_ERR_TIMEOUT, "a grid barrier of the Rayleigh-Ritz eigensolver gave up");
      return BCHDAV_ERR_TIMEOUT;
    }
    if (reinterpret_cast<int*>(hp + act_max)[0] != 0) {
      h->set_error(BCHDAV_ERR_NONFINITE, "Rayleigh-Ritz eigensolver did not converge");
      return BCHDAV_ERR_NONFINITE;
    }
    for (int i = 0; i < k_old; ++i) Dh[i] = hp[i];
    std::vector<double> rel(nt);
    bool finite = true;
    for (int j = 0; j < nt; ++j) {
      double r2 = hp[act_max + 1 + j], v2 = hp[act_max + 1 + nres + j];
      rel[j] = std::sqrt(r2) / std::sqrt(v2);
      if (!std::isfinite(rel[j])) finite = false;
    }
    for (int i = 0; i < k_old; ++i)
      if (!std::isfinite(Dh[i])) finite = false;
    if (!finite) {
      h->set_error(BCHDAV_ERR_NONFINITE, "non-finite Ritz value or residual");
      return BCHDAV_ERR_NONFINITE;
    }
    // convergence + stable partition (converged first)
    std::vector<int> order;
    order.reserve(nt);
    for (int j = 0; j < nt; ++j)
      if (rel[j] <= tol) order.push_back(j);
    const int e_c = (int)order.size();
    for (int j = 0; j < nt; ++j)
      if (!(rel[j] <= tol)) order.push_back(j);
    // mixed path: after a lock, Step 17's next filter inputs reach e_c Ritz vectors beyond the
    // tested block; their float64 residuals are formed now (Ritz values still in Dd), so that
    // every Ritz vector the filter takes is filtered in residual form
    int n_avail = nt;
    if (prec == BCHDAV_PREC_MIXED && e_c > 0) {
      const int n_ext = std::min(e_c, k_act - nt);
      if (n_ext > 0) {
        int np2 = 0;
        tm_res2.start(st);
        if (dd && n_ext % 4 == 0)
          HCUDA(launch_spmm_resid_dd(st, N, A->rowptr, A->colidx, val32, val_lo, V + k_c + nt, ldv,
                                     n_ext, Dd + nt, h->part.as<double>(), &np2,
                                     h->Rres.as<double>() + nt, ldr, negd, dd_scr));
        else
          HCUDA(launch_spmm_resid(st, N, A->rowptr, A->colidx, A->val, V + k_c + nt, ldv, n_ext,
                                  Dd + nt, h->part.as<double>(), &np2, h->Rres.as<double>() + nt,
                                  ldr, negd, h->long_rows()));
        tm_res2.stop(st);
        ++n_spmm;
        n_avail = nt + n_ext;
      }
    }
    bool identity = true;
    for (int j = 0; j < nt; ++j) identity = identity && (order[j] == j);
    if (!identity) {
      int* pi = reinterpret_cast<int*>(hp + 2 * act_max + 2 * ncols + 8);
      for (int j = 0; j < nt; ++j) pi[j] = order[j];
      HCUDA(cudaMemcpyAsync(perm_d, pi, nt * sizeof(int), cudaMemcpyHostToDevice, st));
      double* tmp = h->R.as<double>();
      HCUDA(launch_gather_cols(st, N, nt, V + k_c, ldv, perm_d, tmp, ldb));
      HCUDA(launch_copy_block(st, N, nt, tmp, ldb, V + k_c, ldv));
      std::vector<double> dn(nt);
      for (int j = 0; j < nt; ++j) dn[j] = Dh[order[j]];
      for (int j = 0; j < nt; ++j) Dh[j] = dn[j];
    }
    for (int j = 0; j < e_c; ++j) eval_locked.push_back(Dh[j]);
    k_c += e_c;
    double maxres = 0.0;
    for (double r : rel) maxres = std::max(maxres, r);
    double minres = INFINITY;
    for (double r : rel) minres = std::min(minres, r);
    if (opts.record_history) {
      bchdav_iter_record rec;
      std::memset(&rec, 0, sizeof(rec));
      rec.it = it;
      rec.k_c = k_c;
      rec.e_c = e_c;
      rec.k_act = k_act;
      rec.k_sub = k_sub;
      rec.k_old = k_old;
      rec.n_rep = nrep;
      rec.k_orth = k_orth;
      rec.low_nwb = low_nwb;
      rec.max_resid = maxres;
      rec.min_resid = minres;
      h->history.push_back(rec);
    }
    // Step 13: exit
    if (k_c >= k) {
      converged = true;
      break;
    }
    // Step 14: the converged columns leave the active space
    if (e_c > 0) k_act -= e_c;
    // Step 15: H = diag(non-converged Ritz values)
    std::vector<double> d_act(Dh.begin() + e_c, Dh.begin() + e_c + k_act);
    // Step 16: outer restart
    if (k_sub + b > dim_max) {
      const int k_ro = dim_max - 2 * b - k_c;
      k_act = std::min(k_act, std::max(k_ro, b));
      k_sub = k_c + k_act;
    }
    for (int i = 0; i < (int)d_act.size(); ++i) hp[i] = d_act[i];
    HCUDA(cudaMemcpyAsync(Dd, hp, std::max<size_t>(d_act.size(), 1) * sizeof(double),
                          cudaMemcpyHostToDevice, st));
    HCUDA(launch_h_diag(st, Hm, act_max, Dd, k_act, act_max));
    // Step 17: next filter input
    const int n_i = (k_init > k_i) ? std::min(e_c, k_init - k_i) : 0;
    const int n_r = std::min(b - n_i, k_act);
    const int n_x = b - n_i - n_r;
    if (n_i > 0)
      HCUDA(launch_copy_block(st, N, n_i, opts.v_init + k_i, opts.ld_v_init, Vtmp, ldb));
    if (n_r > 0) HCUDA(launch_copy_block(st, N, n_r, V + k_c, ldv, Vtmp + n_i, ldb));
    for (int j = 0; j < n_x; ++j)
      HCUDA(launch_fill_random_col(st, N, Vtmp, ldb, n_i + n_r + j, opts.seed, kStreamFill,
                                   fill_counter++));
    k_i += n_i;
    for (int j = 0; j < b; ++j) {
      mix_src[j] = -1;
      mix_theta[j] = NAN;
    }
    for (int j = 0; j < n_r; ++j) {
      const int pre = e_c + j;   // position in the active block after the partition
      if (pre < n_avail) {
        mix_src[n_i + j] = pre < nt ? order[pre] : pre;
        mix_theta[n_i + j] = Dh[pre];
      }
    }
    // Step 18: new cut
    if (k_act > 0) {
      std::vector<double> tmpd(d_act.begin(), d_act.begin() + k_act);
      double med = median_of(tmpd);
      if (med > lowb + kLowNwbEps && med < upperb) low_nwb = med;
    }
  }
  HCUDA(cudaStreamSynchronize(st));   // copies queued from host_pinned are complete
  // ---- output: locked pairs sorted ascending (stable), k of them
  const int n_out = std::min<int>(k, (int)eval_locked.size());
  std::vector<int> idx(eval_locked.size());
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int x, int y) { return eval_locked[x] < eval_locked[y]; });
  double max_rel = 0.0;
  if (n_out > 0) {
    int* pi = reinterpret_cast<int*>(hp + 2 * act_max + 2 * ncols + 8);
    double* ev = hp;
    for (int j = 0; j < n_out; ++j) {
      pi[j] = idx[j];
      ev[j] = eval_locked[idx[j]];
    }
    HCUDA(cudaMemcpyAsync(perm_d, pi, n_out * sizeof(int), cudaMemcpyHostToDevice, st));
    HCUDA(cudaMemcpyAsync(evals, ev, n_out * sizeof(double), cudaMemcpyHostToDevice, st));
    HCUDA(launch_gather_cols(st, N, n_out, V, ldv, perm_d, evecs, k));
    // final check: fresh float64 residuals of the returned pairs
    for (int c0 = 0; c0 < n_out; c0 += std::min(64, ldr)) {
      int w = std::min(std::min(64, ldr), n_out - c0);
      int np = 0;
      HCUDA(launch_spmm_resid(st, N, A->rowptr, A->colidx, A->val, evecs + c0, k, w, evals + c0,
                              h->part.as<double>(), &np, h->Rres.as<double>(), ldr, negd,
                              h->long_rows()));
      HCUDA(launch_reduce_partials(st, h->part.as<double>(), np, 2 * w, dsel, 1.0));
      HCUDA(cudaMemcpyAsync(hp + 1024 - 128, dsel, 2 * w * sizeof(double), cudaMemcpyDeviceToHost, st));
      HCUDA(cudaStreamSynchronize(st));
      for (int j = 0; j < w; ++j) {
        double r = std::sqrt(hp[1024 - 128 + j]) / std::sqrt(hp[1024 - 128 + w + j]);
        max_rel = std::max(max_rel, r);
      }
    }
  }
  tm_total.stop(st);
  HCUDA(cudaStreamSynchronize(st));
  collect();
  tm_total.collect();
  if (opts.dense_path == 0) {
    int flag = 0;
    HCUDA(cudaMemcpy(&flag, h->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
      h->set_error(BCHDAV_ERR_TIMEOUT, "solve: a tensor-core wait expired");
      return BCHDAV_ERR_TIMEOUT;
    }
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = it;
    info->n_converged = (int)eval_locked.size();
    info->n_spmm = n_spmm;
    info->n_replaced = n_rep_total;
    info->max_rel_resid = max_rel;
    info->ms_total = tm_total.acc;
    info->ms_filter = tm_filter.acc;
    info->ms_orth = tm_orth.acc;
    info->ms_spmm_w = tm_spmm.acc;
    info->ms_h = tm_h.acc;
    info->ms_eig = tm_eig.acc;
    info->ms_rot = tm_rot.acc;
    info->ms_resid = tm_res.acc + tm_res2.acc;
    info->ms_other = tm_total.acc - (tm_filter.acc + tm_orth.acc + tm_spmm.acc + tm_h.acc +
                                     tm_eig.acc + tm_rot.acc + tm_res.acc + tm_res2.acc);
    info->filter_bytes = filter_bytes;
    info->filter_ms_kernels = tm_filter.acc;
    info->n_kernel_launches =
        (int64_t)(__atomic_load_n(&bchdav::g_launches, __ATOMIC_RELAXED) - launches0);
    info->lowb = lowb;
    info->upperb = upperb;
  }
  return converged ? BCHDAV_OK : BCHDAV_NOT_CONVERGED;
}

bchdav_status bchdav_solve_host(bchdav_handle h, int32_t n, int64_t nnz, const int32_t* rowptr,
                                const int32_t* colidx, const double* val, int32_t k, int32_t b,
                                int32_t m, int32_t act_max, double tol, const bchdav_opts* opts_in,
                                double* evals_host, double* evecs_host, bchdav_info* info) {
  if (!h) return BCHDAV_ERR_ARG;
  if (n < 1 || nnz < n || nnz >= (int64_t)INT32_MAX || !rowptr || !colidx || !val || !evals_host ||
      !evecs_host || k < 1 || k > n) {
    h->set_error(BCHDAV_ERR_ARG, "solve_host: invalid arguments");
    return BCHDAV_ERR_ARG;
  }
  bchdav_opts opts;
  std::memset(&opts, 0, sizeof(opts));
  if (opts_in) opts = *opts_in;
  cudaStream_t st = h->stream;
  BCHDAV_TRY(h->ensure(h->hrow, (size_t)(n + 1) * sizeof(int32_t)));
  BCHDAV_TRY(h->ensure(h->hcol, (size_t)nnz * sizeof(int32_t)));
  BCHDAV_TRY(h->ensure(h->hval, (size_t)nnz * sizeof(double)));
  BCHDAV_TRY(h->ensure(h->hev, (size_t)k * sizeof(double)));
  BCHDAV_TRY(h->ensure(h->hevec, (size_t)n * k * sizeof(double)));
  HCUDA(cudaMemcpyAsync(h->hrow.p, rowptr, (size_t)(n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  HCUDA(cudaMemcpyAsync(h->hcol.p, colidx, (size_t)nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  HCUDA(cudaMemcpyAsync(h->hval.p, val, (size_t)nnz * sizeof(double), cudaMemcpyHostToDevice, st));
  if (opts.k_init > 0 && opts.v_init) {
    BCHDAV_TRY(h->ensure(h->hvinit, (size_t)n * opts.k_init * sizeof(double)));
    if (opts.ld_v_init == opts.k_init)   // contiguous: one linear copy (a pitched copy of
                                         // short rows moves row by row)
      HCUDA(cudaMemcpyAsync(h->hvinit.p, opts.v_init, (size_t)n * opts.k_init * sizeof(double),
                            cudaMemcpyHostToDevice, st));
    else
      HCUDA(cudaMemcpy2DAsync(h->hvinit.p, (size_t)opts.k_init * sizeof(double), opts.v_init,
                              (size_t)opts.ld_v_init * sizeof(double),
                              (size_t)opts.k_init * sizeof(double), (size_t)n,
                              cudaMemcpyHostToDevice, st));
    opts.v_init = h->hvinit.as<double>();
    opts.ld_v_init = opts.k_init;
  }
  bchdav_csr A;
  A.n = n;
  A.nnz = nnz;
  A.rowptr = h->hrow.as<int32_t>();
  A.colidx = h->hcol.as<int32_t>();
  A.val = h->hval.as<double>();
  A.val_f32 = nullptr;
  bchdav_status s = bchdav_solve(h, &A, k, b, m, act_max, tol, &opts, h->hev.as<double>(),
                                 h->hevec.as<double>(), info);
  if (s != BCHDAV_OK && s != BCHDAV_NOT_CONVERGED) return s;
  HCUDA(cudaMemcpyAsync(evals_host, h->hev.p, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, st));
  HCUDA(cudaMemcpyAsync(evecs_host, h->hevec.p, (size_t)n * k * sizeof(double),
                        cudaMemcpyDeviceToHost, st));
  HCUDA(cudaStreamSynchronize(st));
  return s;
}

}  // extern "C"
