// In-block part of the orthonormalisation of Algorithm 2, Step 6: columns of
// the new N x b block are made orthonormal one after another with two
// classical Gram-Schmidt passes against the columns already accepted, and a
// column whose remaining norm is <= tau_dep * (its norm before any
// projection) is reported as numerically dependent (the caller replaces it by
// a random vector, as the paper prescribes, and redoes the block).
//
// One cooperative launch covers all b columns: every pass is "dot products
// (grid reduction) -> update + norm (grid reduction)".  Each thread keeps the
// same rows for the whole launch, so a thread only ever re-reads rows it wrote
// itself; every block reduces the per-block partials in the same fixed order,
// so all blocks take the same decisions and results are bitwise reproducible.
#include <cooperative_groups.h>

#include <algorithm>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace bchdav {

constexpr int kGsThreads = 256;
constexpr int kGsWarps = kGsThreads / 32;

template <int MAXB>
__global__ void __launch_bounds__(kGsThreads) inblock_gs_kernel(
    int n, double* __restrict__ X, int ldx, int b, int j0, const double* __restrict__ norm0,
    double tau_dep, double* __restrict__ red, int* __restrict__ dep,
    double* __restrict__ final_norms) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double s_w[kGsWarps][MAXB];
  __shared__ double s_h[MAXB];
  __shared__ double s_nrm;
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const int G = gridDim.x;
  // red layout: [2 buffers][G][MAXB] dots, then [2][G] norms
  double* dots = red;
  double* nrms = red + 2 * (size_t)G * MAXB;
  const int gtid = blockIdx.x * kGsThreads + t;
  const int gstride = G * kGsThreads;
  int buf = 0;
  for (int j = j0; j < b; ++j) {
    double nrm = 0.0;
    const int npass = (j > 0) ? 2 : 1;
    for (int pass = 0; pass < npass; ++pass) {
      if (j > 0) {
        // ---- dots h_i = x_i^T x_j, i < j
        double part[MAXB];
#pragma unroll
        for (int i = 0; i < MAXB; ++i) part[i] = 0.0;
        for (int r = gtid; r < n; r += gstride) {
          const double* row = X + (size_t)r * ldx;
          double xj = row[j];
#pragma unroll
          for (int i = 0; i < MAXB; ++i)
            if (i < j) part[i] = fma(row[i], xj, part[i]);
        }
#pragma unroll
        for (int i = 0; i < MAXB; ++i) {
          if (i < j) {
            double v = part[i];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) s_w[warp][i] = v;
          }
        }
        __syncthreads();
        if (t < j) {
          double s = 0.0;
          for (int w = 0; w < kGsWarps; ++w) s += s_w[w][t];
          dots[((size_t)buf * G + blockIdx.x) * MAXB + t] = s;
        }
        grid.sync();
        if (t < j) {
          double s = 0.0;
          for (int g = 0; g < G; ++g) s += dots[((size_t)buf * G + g) * MAXB + t];
          s_h[t] = s;
        }
        __syncthreads();
      }
      // ---- update x_j -= sum_i h_i x_i ; norm^2
      double ss = 0.0;
      for (int r = gtid; r < n; r += gstride) {
        double* row = X + (size_t)r * ldx;
        double xj = row[j];
        if (j > 0) {
#pragma unroll
          for (int i = 0; i < MAXB; ++i)
            if (i < j) xj = fma(-s_h[i], row[i], xj);
          row[j] = xj;
        }
        ss = fma(xj, xj, ss);
      }
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
      if (lane == 0) s_w[warp][0] = ss;
      __syncthreads();
      if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kGsWarps; ++w) s += s_w[w][0];
        nrms[(size_t)buf * G + blockIdx.x] = s;
      }
      grid.sync();
      if (t == 0) {
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += nrms[(size_t)buf * G + g];
        s_nrm = sqrt(s);
      }
      __syncthreads();
      nrm = s_nrm;
      buf ^= 1;
    }
    const double n0 = norm0[j];
    if (!(n0 > 0.0) || !(nrm > tau_dep * n0)) {
      if (blockIdx.x == 0 && t == 0) *dep = j;
      return;   // uniform decision: every block reduced the same partials
    }
    if (blockIdx.x == 0 && t == 0) final_norms[j] = nrm;
    const double inv = 1.0 / nrm;
    for (int r = gtid; r < n; r += gstride) X[(size_t)r * ldx + j] *= inv;
  }
}

size_t inblock_gs_scratch_doubles(int b) {
  int maxb = b <= 32 ? 32 : 64;
  return (size_t)2 * (4 * kSMs) * maxb + 2 * (4 * kSMs);
}

template <int MAXB>
static cudaError_t launch_gs(cudaStream_t st, int n, double* X, int ldx, int b, int j0,
                             const double* norm0, double tau_dep, double* scratch, int* dep,
                             double* final_norms, int grid_cap) {
  // co-resident blocks, at most 4 per SM (thread-safe static initialisation)
  static const int wave = []() {
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, inblock_gs_kernel<MAXB>,
                                                      kGsThreads, 0) != cudaSuccess) {
      cudaGetLastError();
      return 1;
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, std::min(per_sm, 4) * sms);
  }();
  int grid = wave;
  int need = ceil_div(n, kGsThreads);
  if (grid > need) grid = need;
  if (grid > 4 * kSMs) grid = 4 * kSMs;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  if (grid < 1) grid = 1;
  void* args[] = {&n, &X, &ldx, &b, &j0, &norm0, &tau_dep, &scratch, &dep, &final_norms};
  note_launch();
  return cudaLaunchCooperativeKernel((const void*)inblock_gs_kernel<MAXB>, grid, kGsThreads, args,
                                     0, st);
}

cudaError_t launch_inblock_gs(cudaStream_t st, int n, double* X, int ldx, int b, int j0,
                              const double* norm0, double tau_dep, double* scratch, int* dep,
                              double* final_norms, int grid_cap) {
  if (b <= 0 || b > 64) return cudaErrorInvalidValue;
  if (b <= 32)
    return launch_gs<32>(st, n, X, ldx, b, j0, norm0, tau_dep, scratch, dep, final_norms,
                         grid_cap);
  return launch_gs<64>(st, n, X, ldx, b, j0, norm0, tau_dep, scratch, dep, final_norms, grid_cap);
}

}  // namespace bchdav
