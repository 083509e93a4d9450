// Eq. (1) on the device: A = I - D^{-1/2} S D^{-1/2} from an undirected edge
// list, in canonical CSR (columns ascending, explicit unit diagonal,
// off-diagonal -(r_i * r_j) with r_i = 1/sqrt(d_i) rounded per IEEE).
//
// 1. count both orientations of every non-loop edge per row (atomics);
// 2. exclusive scan -> row segments; scatter the neighbours (atomics: the
//    order inside a row is arbitrary at this point);
// 3. sort every row segment (bitonic: in shared memory for rows up to 4096
//    entries, in global memory for longer rows, all long rows per launch) and
//    count distinct neighbours -> degree d_i;
// 4. exclusive scan of (d_i + 1) -> rowptr; r_i = 1/sqrt(d_i);
// 5. one warp per row writes the distinct neighbours and the diagonal in
//    ascending order with their values (float64 and its float32 rounding).
// Sorting makes the result independent of the atomic order: the CSR is
// bitwise deterministic.
#include <algorithm>
#include <cstring>
#include <vector>

#include "handle.cuh"
#include "kernels.cuh"

using namespace bchdav;

namespace {

constexpr int kSortSmem = 4096;   // rows up to this length are sorted in shared memory

__global__ void count_kernel(long long ne, const int* __restrict__ src, const int* __restrict__ dst,
                             int n, int* __restrict__ cnt, int* __restrict__ bad) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    int u = src[e], v = dst[e];
    if (u < 0 || u >= n || v < 0 || v >= n) {
      atomicOr(bad, 1);
      continue;
    }
    if (u == v) continue;
    atomicAdd(cnt + u, 1);
    atomicAdd(cnt + v, 1);
  }
}

}  // namespace

// ---- exclusive scan of int counts into int64 offsets (three phases); also used by the SpMM
// long-row schedule
namespace bchdav {
constexpr int kScanTile = 2048;

__global__ void scan_tiles_kernel(int n, const int* __restrict__ in, int add_one,
                                  long long* __restrict__ out, long long* __restrict__ tile_sums) {
  __shared__ long long s[kScanTile];
  const int base = blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
    int g = base + i;
    s[i] = (g < n) ? (long long)in[g] + add_one : 0;
  }
  __syncthreads();
  // Hillis-Steele is O(n log n) work but the tile is small; use a simple up-sweep/down-sweep
  for (int off = 1; off < kScanTile; off <<= 1) {
    for (int i = threadIdx.x; i < kScanTile / (2 * off); i += blockDim.x) {
      int idx = (i + 1) * off * 2 - 1;
      s[idx] += s[idx - off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    tile_sums[blockIdx.x] = s[kScanTile - 1];
    s[kScanTile - 1] = 0;
  }
  __syncthreads();
  for (int off = kScanTile / 2; off >= 1; off >>= 1) {
    for (int i = threadIdx.x; i < kScanTile / (2 * off); i += blockDim.x) {
      int idx = (i + 1) * off * 2 - 1;
      long long tmp = s[idx - off];
      s[idx - off] = s[idx];
      s[idx] += tmp;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
    int g = base + i;
    if (g < n) out[g] = s[i];
  }
}

__global__ void scan_sums_kernel(int ntiles, long long* __restrict__ tile_sums,
                                 long long* __restrict__ total) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    long long run = 0;
    for (int i = 0; i < ntiles; ++i) {
      long long v = tile_sums[i];
      tile_sums[i] = run;
      run += v;
    }
    *total = run;
  }
}

__global__ void scan_add_kernel(int n, long long* __restrict__ out,
                                const long long* __restrict__ tile_sums,
                                const long long* __restrict__ total) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g <= n;
       g += (long long)gridDim.x * blockDim.x) {
    if (g == n) out[n] = *total;
    else out[g] += tile_sums[g / kScanTile];
  }
}

cudaError_t exclusive_scan(cudaStream_t st, int n, const int* in, int add_one, long long* out,
                           long long* tile_sums) {
  int ntiles = ceil_div(n, kScanTile);
  scan_tiles_kernel<<<ntiles, 512, 0, st>>>(n, in, add_one, out, tile_sums); note_launch();
  scan_sums_kernel<<<1, 32, 0, st>>>(ntiles, tile_sums, tile_sums + ntiles); note_launch();
  scan_add_kernel<<<ceil_div(n + 1, 256) < 4096 ? ceil_div(n + 1, 256) : 4096, 256, 0, st>>>(
      n, out, tile_sums, tile_sums + ntiles); note_launch();
  return cudaGetLastError();
}

}  // namespace bchdav

namespace {

__global__ void scatter_kernel(long long ne, const int* __restrict__ src, const int* __restrict__ dst,
                               const long long* __restrict__ start, int* __restrict__ fill,
                               int* __restrict__ adj) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    int u = src[e], v = dst[e];
    if (u == v) continue;
    adj[start[u] + atomicAdd(fill + u, 1)] = v;
    adj[start[v] + atomicAdd(fill + v, 1)] = u;
  }
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// One block per row of length <= kSortSmem: bitonic sort in shared memory,
// write back sorted, count distinct entries.
__global__ void __launch_bounds__(256) sort_rows_smem_kernel(int n, const long long* __restrict__ start,
                                                             int* __restrict__ adj,
                                                             int* __restrict__ deg,
                                                             int* __restrict__ long_rows,
                                                             int* __restrict__ n_long) {
  __shared__ int s[kSortSmem];
  __shared__ int s_cnt[8];
  for (int row = blockIdx.x; row < n; row += gridDim.x) {
    const long long b0 = start[row];
    const int len = (int)(start[row + 1] - b0);
    if (len > kSortSmem) {
      if (threadIdx.x == 0) {
        long_rows[atomicAdd(n_long, 1)] = row;
        deg[row] = -1;
      }
      continue;
    }
    if (len <= 1) {
      if (threadIdx.x == 0) deg[row] = len;
      continue;
    }
    const int P = next_pow2(len);
    for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = (i < len) ? adj[b0 + i] : INT_MAX;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
          int p = i ^ j;
          if (p > i) {
            int a = s[i], c = s[p];
            bool up = ((i & k) == 0);
            if ((a > c) == up) {
              s[i] = c;
              s[p] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    int cnt = 0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      adj[b0 + i] = s[i];
      cnt += (i == 0 || s[i] != s[i - 1]);
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_cnt[w];
      deg[row] = t;
    }
    __syncthreads();
  }
}

// Long rows: copy into power-of-two padded segments of a scratch array.
__global__ void long_copy_kernel(int nl, const int* __restrict__ rows, const long long* __restrict__ start,
                                 const long long* __restrict__ seg, const int* __restrict__ adj,
                                 int* __restrict__ scratch, int to_scratch) {
  const int r = blockIdx.y;
  if (r >= nl) return;
  const int row = rows[r];
  const long long b0 = start[row];
  const int len = (int)(start[row + 1] - b0);
  const long long s0 = seg[r];
  const long long P = seg[r + 1] - s0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    if (to_scratch) scratch[s0 + i] = (i < len) ? adj[b0 + i] : INT_MAX;
    else if (i < len) const_cast<int*>(adj)[b0 + i] = scratch[s0 + i];
  }
}

// One bitonic stage (k, j) on every long segment whose size is >= k.
__global__ void long_stage_kernel(int nl, const long long* __restrict__ seg, int* __restrict__ a,
                                  long long k, long long j) {
  const int r = blockIdx.y;
  if (r >= nl) return;
  const long long s0 = seg[r];
  const long long P = seg[r + 1] - s0;
  if (k > P) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    long long p = i ^ j;
    if (p > i) {
      int x = a[s0 + i], y = a[s0 + p];
      bool up = ((i & k) == 0);
      if ((x > y) == up) {
        a[s0 + i] = y;
        a[s0 + p] = x;
      }
    }
  }
}

__global__ void long_count_kernel(int nl, const int* __restrict__ rows, const long long* __restrict__ start,
                                  const int* __restrict__ adj, int* __restrict__ deg) {
  __shared__ int s_cnt[8];
  const int r = blockIdx.x;
  if (r >= nl) return;
  const int row = rows[r];
  const long long b0 = start[row];
  const int len = (int)(start[row + 1] - b0);
  int cnt = 0;
  for (int i = threadIdx.x; i < len; i += blockDim.x)
    cnt += (i == 0 || adj[b0 + i] != adj[b0 + i - 1]);
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_cnt[w];
    deg[row] = t;
  }
}

// r_i = 1/sqrt(d_i) (0 for an isolated node) for Eq. (1); d_i itself for L = D - S
__global__ void rsqrt_deg_kernel(int n, const int* __restrict__ deg, double* __restrict__ r,
                                 int kind) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int d = deg[i];
    r[i] = kind == BCHDAV_LAPLACIAN_COMBINATORIAL ? (double)d
                                                  : (d > 0 ? 1.0 / sqrt((double)d) : 0.0);
  }
}

// One warp per row: distinct neighbours plus the diagonal, ascending.  Eq. (1): off-diagonal
// -(r_i r_j), diagonal 1; L = D - S: off-diagonal -1, diagonal d_i (r_i holds d_i).
__global__ void fill_kernel(int n, const long long* __restrict__ start, const int* __restrict__ adj,
                            const long long* __restrict__ rowptr64, const double* __restrict__ r,
                            int* __restrict__ rowptr, int* __restrict__ colidx,
                            double* __restrict__ val, float* __restrict__ val32, int kind) {
  const bool comb = kind == BCHDAV_LAPLACIAN_COMBINATORIAL;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += warps) {
    const long long b0 = start[row];
    const int len = (int)(start[row + 1] - b0);
    const long long o0 = rowptr64[row];
    if (lane == 0) {
      rowptr[row] = (int)o0;
      if (row == n - 1) rowptr[n] = (int)rowptr64[n];
    }
    const double ri = r[row];
    int written = 0;   // distinct entries emitted so far
    int below = 0;     // distinct entries < row
    for (int c0 = 0; c0 < len; c0 += 32) {
      const int i = c0 + lane;
      int v = 0;
      bool uniq = false;
      if (i < len) {
        v = adj[b0 + i];
        uniq = (i == 0) || (adj[b0 + i - 1] != v);
      }
      unsigned m = __ballot_sync(0xffffffffu, uniq);
      unsigned mb = __ballot_sync(0xffffffffu, uniq && v < row);
      if (uniq) {
        int rank = written + __popc(m & ((1u << lane) - 1u));
        long long pos = o0 + rank + (v > row ? 1 : 0);
        double x = comb ? -1.0 : -(ri * r[v]);
        colidx[pos] = v;
        val[pos] = x;
        val32[pos] = __double2float_rn(x);
      }
      written += __popc(m);
      below += __popc(mb);
    }
    if (lane == 0) {
      long long pos = o0 + below;
      colidx[pos] = row;
      val[pos] = comb ? ri : 1.0;
      val32[pos] = comb ? __double2float_rn(ri) : 1.0f;
    }
  }
}

__global__ void check_csr_kernel(int n, long long nnz, const int* __restrict__ rowptr,
                                 const int* __restrict__ colidx, int* __restrict__ bad) {
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
    int a = rowptr[row], b = rowptr[row + 1];
    if (row == 0 && a != 0) atomicOr(bad, 1);
    if (row == n - 1 && (long long)b != nnz) atomicOr(bad, 2);
    if (b < a) {
      atomicOr(bad, 4);
      continue;
    }
    int prev = -1;
    for (int k = a; k < b; ++k) {
      int c = colidx[k];
      if (c < 0 || c >= n) atomicOr(bad, 8);
      if (c <= prev) atomicOr(bad, 16);
      prev = c;
    }
  }
}

int grid_for(long long work) {
  long long g = (work + 255) / 256;
  if (g > 16 * kSMs) g = 16 * kSMs;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

#define HCUDA(expr) BCHDAV_CUDA_OK(expr, h)

extern "C" bchdav_status bchdav_check_csr(bchdav_handle h, const bchdav_csr* A) {
  if (!h) return BCHDAV_ERR_ARG;
  if (!A || A->n <= 0 || !A->rowptr || !A->colidx || A->nnz < 0) {
    h->set_error(BCHDAV_ERR_ARG, "check_csr: invalid descriptor");
    return BCHDAV_ERR_ARG;
  }
  int* bad = nullptr;
  HCUDA(cudaMallocAsync(&bad, sizeof(int), h->stream));
  HCUDA(cudaMemsetAsync(bad, 0, sizeof(int), h->stream));
  check_csr_kernel<<<grid_for(A->n), 256, 0, h->stream>>>(A->n, A->nnz, A->rowptr, A->colidx, bad); note_launch();
  HCUDA(cudaGetLastError());
  int hb = 0;
  HCUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HCUDA(cudaFreeAsync(bad, h->stream));
  HCUDA(cudaStreamSynchronize(h->stream));
  if (hb) {
    h->set_error(BCHDAV_ERR_CSR, "CSR check failed (flags " + std::to_string(hb) + ")");
    return BCHDAV_ERR_CSR;
  }
  return BCHDAV_OK;
}

extern "C" bchdav_status bchdav_free_csr(bchdav_handle h, bchdav_csr* csr) {
  if (!h || !csr) return BCHDAV_ERR_ARG;
  cudaStreamSynchronize(h->stream);
  cudaFree(const_cast<int32_t*>(csr->rowptr));
  cudaFree(const_cast<int32_t*>(csr->colidx));
  cudaFree(const_cast<double*>(csr->val));
  cudaFree(const_cast<float*>(csr->val_f32));
  csr->rowptr = nullptr;
  csr->colidx = nullptr;
  csr->val = nullptr;
  csr->val_f32 = nullptr;
  csr->n = 0;
  csr->nnz = 0;
  return BCHDAV_OK;
}

extern "C" bchdav_status bchdav_copy_csr(bchdav_handle h, const bchdav_csr* csr, int32_t* rowptr,
                                         int32_t* colidx, double* val, float* val_f32) {
  if (!h) return BCHDAV_ERR_ARG;
  if (!csr || !csr->rowptr || !csr->colidx || !csr->val || !rowptr || !colidx || !val ||
      (val_f32 && !csr->val_f32)) {
    h->set_error(BCHDAV_ERR_ARG, "copy_csr: invalid arguments");
    return BCHDAV_ERR_ARG;
  }
  cudaStream_t st = h->stream;
  const size_t nnz = (size_t)csr->nnz;
  HCUDA(cudaMemcpyAsync(rowptr, csr->rowptr, (size_t)(csr->n + 1) * sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, st));
  HCUDA(cudaMemcpyAsync(colidx, csr->colidx, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  HCUDA(cudaMemcpyAsync(val, csr->val, nnz * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (val_f32)
    HCUDA(cudaMemcpyAsync(val_f32, csr->val_f32, nnz * sizeof(float), cudaMemcpyDeviceToDevice, st));
  HCUDA(cudaStreamSynchronize(st));
  return BCHDAV_OK;
}

extern "C" bchdav_status bchdav_build_laplacian(bchdav_handle h, int32_t n, int64_t n_edges,
                                                const int32_t* src, const int32_t* dst,
                                                bchdav_csr* out) {
  return bchdav_build_laplacian_kind(h, n, n_edges, src, dst, BCHDAV_LAPLACIAN_NORMALIZED, out);
}

extern "C" bchdav_status bchdav_build_laplacian_kind(bchdav_handle h, int32_t n, int64_t n_edges,
                                                     const int32_t* src, const int32_t* dst,
                                                     int32_t kind, bchdav_csr* out) {
  if (!h) return BCHDAV_ERR_ARG;
  if (n < 1 || n_edges < 0 || (n_edges > 0 && (!src || !dst)) || !out ||
      2 * n_edges + n >= (int64_t)INT32_MAX ||
      (kind != BCHDAV_LAPLACIAN_NORMALIZED && kind != BCHDAV_LAPLACIAN_COMBINATORIAL)) {
    h->set_error(BCHDAV_ERR_ARG, "build_laplacian: invalid arguments");
    return BCHDAV_ERR_ARG;
  }
  cudaStream_t st = h->stream;
  std::memset(out, 0, sizeof(*out));
  const int ntiles = ceil_div(n + 1, kScanTile);
  // temporaries
  int *cnt = nullptr, *fill = nullptr, *adj = nullptr, *deg = nullptr, *flags = nullptr,
      *long_rows = nullptr;
  long long *start = nullptr, *rp64 = nullptr, *tiles = nullptr;
  double* r = nullptr;
  struct Free {
    std::vector<void*> ptrs;
    ~Free() {
      for (void* p : ptrs) cudaFree(p);
    }
  } fr;
  auto alloc = [&](void** p, size_t bytes) -> bchdav_status {
    cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->set_error(BCHDAV_ERR_OOM, "build_laplacian: allocation failed");
      return BCHDAV_ERR_OOM;
    }
    fr.ptrs.push_back(*p);
    return BCHDAV_OK;
  };
  BCHDAV_TRY(alloc((void**)&cnt, (size_t)n * sizeof(int)));
  BCHDAV_TRY(alloc((void**)&fill, (size_t)n * sizeof(int)));
  BCHDAV_TRY(alloc((void**)&deg, (size_t)n * sizeof(int)));
  BCHDAV_TRY(alloc((void**)&long_rows, (size_t)n * sizeof(int)));
  BCHDAV_TRY(alloc((void**)&flags, 4 * sizeof(int)));
  BCHDAV_TRY(alloc((void**)&start, (size_t)(n + 1) * sizeof(long long)));
  BCHDAV_TRY(alloc((void**)&rp64, (size_t)(n + 1) * sizeof(long long)));
  BCHDAV_TRY(alloc((void**)&tiles, (size_t)(ntiles + 2) * sizeof(long long)));
  BCHDAV_TRY(alloc((void**)&r, (size_t)n * sizeof(double)));
  HCUDA(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int), st));
  HCUDA(cudaMemsetAsync(fill, 0, (size_t)n * sizeof(int), st));
  HCUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
  if (n_edges > 0) {
    count_kernel<<<grid_for(n_edges), 256, 0, st>>>(n_edges, src, dst, n, cnt, flags); note_launch();
    HCUDA(cudaGetLastError());
  }
  int hflags[4] = {0, 0, 0, 0};
  HCUDA(cudaMemcpyAsync(hflags, flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  HCUDA(cudaStreamSynchronize(st));
  if (hflags[0]) {
    h->set_error(BCHDAV_ERR_ARG, "build_laplacian: edge endpoint outside [0, n)");
    return BCHDAV_ERR_ARG;
  }
  HCUDA(exclusive_scan(st, n, cnt, 0, start, tiles));
  long long total = 0;
  HCUDA(cudaMemcpyAsync(&total, start + n, sizeof(long long), cudaMemcpyDeviceToHost, st));
  HCUDA(cudaStreamSynchronize(st));
  BCHDAV_TRY(alloc((void**)&adj, (size_t)(total > 0 ? total : 1) * sizeof(int)));
  if (n_edges > 0) {
    scatter_kernel<<<grid_for(n_edges), 256, 0, st>>>(n_edges, src, dst, start, fill, adj); note_launch();
    HCUDA(cudaGetLastError());
  }
  // sort rows
  sort_rows_smem_kernel<<<n < 16 * kSMs * 8 ? n : 16 * kSMs * 8, 256, 0, st>>>(n, start, adj, deg,
                                                                              long_rows, flags + 1); note_launch();
  HCUDA(cudaGetLastError());
  int n_long = 0;
  HCUDA(cudaMemcpyAsync(&n_long, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  HCUDA(cudaStreamSynchronize(st));
  if (n_long > 0) {
    // sort the long-row list so that the scratch layout is deterministic
    std::vector<int> lr(n_long);
    HCUDA(cudaMemcpy(lr.data(), long_rows, n_long * sizeof(int), cudaMemcpyDeviceToHost));
    std::sort(lr.begin(), lr.end());
    std::vector<long long> hstart(n_long), hend(n_long);
    std::vector<long long> seg(n_long + 1, 0);
    long long maxP = 1;
    for (int i = 0; i < n_long; ++i) {
      long long b0, b1;
      HCUDA(cudaMemcpy(&b0, start + lr[i], sizeof(long long), cudaMemcpyDeviceToHost));
      HCUDA(cudaMemcpy(&b1, start + lr[i] + 1, sizeof(long long), cudaMemcpyDeviceToHost));
      long long len = b1 - b0, P = 1;
      while (P < len) P <<= 1;
      seg[i + 1] = seg[i] + P;
      maxP = P > maxP ? P : maxP;
    }
    long long* seg_d = nullptr;
    int* scratch = nullptr;
    BCHDAV_TRY(alloc((void**)&seg_d, (n_long + 1) * sizeof(long long)));
    BCHDAV_TRY(alloc((void**)&scratch, (size_t)seg[n_long] * sizeof(int)));
    HCUDA(cudaMemcpy(long_rows, lr.data(), n_long * sizeof(int), cudaMemcpyHostToDevice));
    HCUDA(cudaMemcpy(seg_d, seg.data(), (n_long + 1) * sizeof(long long), cudaMemcpyHostToDevice));
    dim3 g((unsigned)std::min<long long>((maxP + 255) / 256, 1024), (unsigned)n_long);
    long_copy_kernel<<<g, 256, 0, st>>>(n_long, long_rows, start, seg_d, adj, scratch, 1); note_launch();
    for (long long k = 2; k <= maxP; k <<= 1)
      for (long long j = k >> 1; j > 0; j >>= 1)
        long_stage_kernel<<<g, 256, 0, st>>>(n_long, seg_d, scratch, k, j); note_launch();
    long_copy_kernel<<<g, 256, 0, st>>>(n_long, long_rows, start, seg_d, adj, scratch, 0); note_launch();
    long_count_kernel<<<n_long, 256, 0, st>>>(n_long, long_rows, start, adj, deg); note_launch();
    HCUDA(cudaGetLastError());
  }
  // rowptr from (d_i + 1), r_i = 1/sqrt(d_i)
  HCUDA(exclusive_scan(st, n, deg, 1, rp64, tiles));
  long long nnz = 0;
  HCUDA(cudaMemcpyAsync(&nnz, rp64 + n, sizeof(long long), cudaMemcpyDeviceToHost, st));
  rsqrt_deg_kernel<<<grid_for(n), 256, 0, st>>>(n, deg, r, kind); note_launch();
  HCUDA(cudaGetLastError());
  HCUDA(cudaStreamSynchronize(st));
  int32_t* rowptr = nullptr;
  int32_t* colidx = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;
  if (cudaMalloc(&rowptr, (size_t)(n + 1) * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&colidx, (size_t)nnz * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&val, (size_t)nnz * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&val32, (size_t)nnz * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(rowptr);
    cudaFree(colidx);
    cudaFree(val);
    cudaFree(val32);
    h->set_error(BCHDAV_ERR_OOM, "build_laplacian: output allocation failed");
    return BCHDAV_ERR_OOM;
  }
  fill_kernel<<<grid_for((long long)n * 32), 256, 0, st>>>(n, start, adj, rp64, r, rowptr, colidx,
                                                          val, val32, kind); note_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(rowptr);
    cudaFree(colidx);
    cudaFree(val);
    cudaFree(val32);
    h->set_error(BCHDAV_ERR_CUDA, std::string("build_laplacian: ") + cudaGetErrorString(e));
    return BCHDAV_ERR_CUDA;
  }
  out->n = n;
  out->nnz = nnz;
  out->rowptr = rowptr;
  out->colidx = colidx;
  out->val = val;
  out->val_f32 = val32;
  return BCHDAV_OK;
}
