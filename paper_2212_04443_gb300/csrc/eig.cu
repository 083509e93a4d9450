// Step 9 of Algorithm 2: H Y = Y D for the small symmetric Rayleigh-quotient
// matrix H (n <= act_max), in float64, on the device.
//
// Householder reduction to tridiagonal form (P_k = I - 2 v v^T, applied as
// A <- A - 2 (v w^T + w v^T) with w = A v - (v^T A v) v), backward accumulation
// of Q = P_0 ... P_{n-3}, then the implicitly shifted QL iteration on the
// tridiagonal matrix (Bowdler, Martin, Reinsch, Wilkinson 1968) with each
// sweep's plane rotations recorded by one thread and applied to the rows of
// (QZ)^T by all threads in parallel.  Eigenvalues are returned ascending.
#include <mutex>

#include "kernels.cuh"

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
