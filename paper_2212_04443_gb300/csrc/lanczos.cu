// Spectrum bounds by k-step Lanczos (Sec. 2: the filter's bounds are analytic for the
// normalized Laplacian and otherwise estimated by standard Lanczos with a few matrix-vector
// products; the estimator is the one of the Chebyshev-Davidson work the paper cites, Zhou and
// Li 2011).
//
//   v_1 = u / ||u||, u_i = Philox stream 3, vector 0, row i (uniform in [-1/2, 1/2))
//   for j = 1..k:  w = A v_j - beta_{j-1} v_{j-1};  alpha_j = v_j . w;  w = w - alpha_j v_j;
//                  beta_j = ||w||;  v_{j+1} = w / beta_j
//   T_k = tridiag(beta; alpha; beta), theta its eigenvalues:
//   upperb = theta_max + beta_k (the residual norm of A V_k = V_k T_k + f_k e_k^T),
//   lowb = theta_min.
// An exactly zero beta_j (an invariant subspace) ends the recurrence after step j.
// The matrix-vector product is the filter's row SpMM with one column; dot products and norms
// are two-stage sums in a fixed order (deterministic); the k x k eigenvalue problem runs on the
// device eigensolver.
#include <cmath>
#include <vector>

#include "handle.cuh"

namespace bchdav {
namespace {

constexpr int kLzThreads = 256;
constexpr int kLzMaxSteps = 64;

__device__ __forceinline__ double lz_block_sum(double v, double* s) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) s[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s[i];
  return t;   // valid in thread 0
}

// u (the unnormalised start vector) and per-CTA partial sums of u_i^2
__global__ void lz_start_kernel(int n, unsigned long long seed, double* __restrict__ v,
                                double* __restrict__ partial) {
  __shared__ double s[kLzThreads / 32];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double u = philox_pm_half(seed, kStreamLanczos, 0u, (uint32_t)i);
    v[i] = u;
    acc += u * u;
  }
  const double t = lz_block_sum(acc, s);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// w <- w - beta_prev v_prev (beta_prev NULL: first step); partial sums of v_i w_i
__global__ void lz_dot_kernel(int n, double* __restrict__ w, const double* __restrict__ v,
                              const double* __restrict__ vp, const double* __restrict__ beta_prev,
                              double* __restrict__ partial) {
  __shared__ double s[kLzThreads / 32];
  const double bp = beta_prev ? *beta_prev : 0.0;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double wi = w[i];
    if (beta_prev) {
      wi -= bp * vp[i];
      w[i] = wi;
    }
    acc += v[i] * wi;
  }
  const double t = lz_block_sum(acc, s);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// w <- w - alpha v; partial sums of w_i^2
__global__ void lz_norm_kernel(int n, double* __restrict__ w, const double* __restrict__ v,
                               const double* __restrict__ alpha, double* __restrict__ partial) {
  __shared__ double s[kLzThreads / 32];
  const double a = *alpha;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double wi = w[i] - a * v[i];
    w[i] = wi;
    acc += wi * wi;
  }
  const double t = lz_block_sum(acc, s);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// out = sum of the partials (fixed order), or its square root
__global__ void lz_finish_kernel(const double* __restrict__ partial, int parts,
                                 double* __restrict__ out, int take_sqrt) {
  __shared__ double s[kLzThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < parts; i += blockDim.x) acc += partial[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = take_sqrt ? sqrt(s[0]) : s[0];
}

// x <- x / *nrm (zero when *nrm is zero)
__global__ void lz_scale_kernel(int n, double* __restrict__ x, const double* __restrict__ nrm) {
  const double d = *nrm;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] = d > 0.0 ? x[i] / d : 0.0;
}

// T (k x k, row-major) from alpha[0..k-1] and beta[0..k-2]
__global__ void lz_tridiag_kernel(int k, const double* __restrict__ alpha,
                                  const double* __restrict__ beta, double* __restrict__ T) {
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e - i * k;
    T[e] = i == j ? alpha[i] : (j == i + 1 ? beta[i] : (i == j + 1 ? beta[j] : 0.0));
  }
}

#define HCUDA(expr) BCHDAV_CUDA_OK(expr, h)

}  // namespace

bchdav_status lanczos_bounds(bchdav_handle h, const bchdav_csr* A, int steps,
                             unsigned long long seed, double* lowb, double* upperb,
                             double* alpha_out, double* beta_out, int* steps_done) {
  const int n = A->n;
  if (steps < 1 || steps > kLzMaxSteps || steps > n) {
    h->set_error(BCHDAV_ERR_ARG, "lanczos_bounds: need 1 <= steps <= min(64, n)");
    return BCHDAV_ERR_ARG;
  }
  cudaStream_t st = h->stream;
  BCHDAV_TRY(prepare_long_rows(h, A, (size_t)64 * sizeof(double)));
  const int grid = std::max(1, std::min(ceil_div(n, kLzThreads), 2 * h->sms));
  const size_t ew = eigh_work_doubles(steps);
  const size_t doubles = 3 * (size_t)n + (size_t)grid + 2 * kLzMaxSteps + 8 +
                         2 * (size_t)steps * steps + steps + ew + 8;
  BCHDAV_TRY(h->ensure(h->lz, doubles * sizeof(double)));
  double* buf[3];
  buf[0] = h->lz.as<double>();
  buf[1] = buf[0] + n;
  buf[2] = buf[1] + n;
  double* partial = buf[2] + n;
  double* alpha = partial + grid;
  double* beta = alpha + kLzMaxSteps;
  double* scal = beta + kLzMaxSteps;   // start-vector norm
  double* T = scal + 8;
  double* Y = T + (size_t)steps * steps;
  double* D = Y + (size_t)steps * steps;
  double* work = D + steps;
  int* status = reinterpret_cast<int*>(work + ew);
  double *vp = buf[0], *v = buf[1], *w = buf[2];

  lz_start_kernel<<<grid, kLzThreads, 0, st>>>(n, seed, v, partial); note_launch();
  lz_finish_kernel<<<1, kLzThreads, 0, st>>>(partial, grid, scal, 1); note_launch();
  lz_scale_kernel<<<grid, kLzThreads, 0, st>>>(n, v, scal); note_launch();
  HCUDA(cudaGetLastError());
  for (int j = 0; j < steps; ++j) {
    HCUDA(launch_spmm_axpby<double>(st, n, A->rowptr, A->colidx, A->val, v, 1, 1, w, 1, nullptr,
                                    0, 1.0, 0.0, 0.0, nullptr, 0, nullptr, h->long_rows()));
    lz_dot_kernel<<<grid, kLzThreads, 0, st>>>(n, w, v, vp, j > 0 ? beta + j - 1 : nullptr,
                                               partial); note_launch();
    lz_finish_kernel<<<1, kLzThreads, 0, st>>>(partial, grid, alpha + j, 0); note_launch();
    lz_norm_kernel<<<grid, kLzThreads, 0, st>>>(n, w, v, alpha + j, partial); note_launch();
    lz_finish_kernel<<<1, kLzThreads, 0, st>>>(partial, grid, beta + j, 1); note_launch();
    lz_scale_kernel<<<grid, kLzThreads, 0, st>>>(n, w, beta + j); note_launch();
    HCUDA(cudaGetLastError());
    double* t = vp;
    vp = v;
    v = w;
    w = t;
  }
  std::vector<double> ab(2 * (size_t)steps);
  HCUDA(cudaMemcpyAsync(ab.data(), alpha, steps * sizeof(double), cudaMemcpyDeviceToHost, st));
  HCUDA(cudaMemcpyAsync(ab.data() + steps, beta, steps * sizeof(double), cudaMemcpyDeviceToHost,
                        st));
  HCUDA(cudaStreamSynchronize(st));
  int k = steps;
  for (int j = 0; j < steps; ++j)
    if (ab[steps + j] == 0.0) {
      k = j + 1;
      break;
    }
  for (int j = 0; j < k; ++j)
    if (!std::isfinite(ab[j]) || !std::isfinite(ab[steps + j])) {
      h->set_error(BCHDAV_ERR_NONFINITE, "lanczos_bounds: non-finite recurrence coefficient");
      return BCHDAV_ERR_NONFINITE;
    }
  lz_tridiag_kernel<<<1, kLzThreads, 0, st>>>(k, alpha, beta, T); note_launch();
  HCUDA(cudaGetLastError());
  HCUDA(launch_eigh(st, k, T, k, D, Y, k, work, status));
  std::vector<double> theta(k);
  int hst = 0;
  HCUDA(cudaMemcpyAsync(theta.data(), D, k * sizeof(double), cudaMemcpyDeviceToHost, st));
  HCUDA(cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  HCUDA(cudaStreamSynchronize(st));
  if (hst != 0) {
    h->set_error(BCHDAV_ERR_NONFINITE, "lanczos_bounds: tridiagonal eigensolver failed");
    return BCHDAV_ERR_NONFINITE;
  }
  *lowb = theta[0];
  *upperb = theta[k - 1] + ab[steps + k - 1];
  if (alpha_out)
    for (int j = 0; j < k; ++j) alpha_out[j] = ab[j];
  if (beta_out)
    for (int j = 0; j < k; ++j) beta_out[j] = ab[steps + j];
  if (steps_done) *steps_done = k;
  return BCHDAV_OK;
}

}  // namespace bchdav

extern "C" bchdav_status bchdav_lanczos_bounds(bchdav_handle h, const bchdav_csr* A,
                                               int32_t steps, uint64_t seed, double* lowb,
                                               double* upperb, double* alpha, double* beta,
                                               int32_t* steps_done) {
  if (!h) return BCHDAV_ERR_ARG;
  if (!A || !A->rowptr || !A->colidx || !A->val || A->n < 1 || !lowb || !upperb) {
    h->set_error(BCHDAV_ERR_ARG, "lanczos_bounds: invalid arguments");
    return BCHDAV_ERR_ARG;
  }
  int done = 0;
  bchdav_status s = bchdav::lanczos_bounds(h, A, steps, seed, lowb, upperb, alpha, beta, &done);
  if (s == BCHDAV_OK && steps_done) *steps_done = done;
  return s;
}
