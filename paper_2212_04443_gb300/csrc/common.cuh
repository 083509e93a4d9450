// Shared device/host helpers of the GB300 block Chebyshev-Davidson library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/bchdav.h"

namespace bchdav {

constexpr int kSMs = 152;   // GB300: 2 dies x 76 SMs (queried at runtime; this is the fallback)

struct Error {
  bchdav_status st;
  std::string msg;
};

// Throw-free error plumbing: functions return bchdav_status; the last message
// is kept in the handle.
#define BCHDAV_CUDA_OK(expr, ctx)                                                   \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) {                                                        \
      (ctx)->set_error(BCHDAV_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
      return BCHDAV_ERR_CUDA;                                                       \
    }                                                                               \
  } while (0)

#define BCHDAV_TRY(expr)                 \
  do {                                   \
    bchdav_status _s = (expr);           \
    if (_s != BCHDAV_OK) return _s;      \
  } while (0)

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
inline int round_up(int a, int m) { return (a + m - 1) / m * m; }

// ---- Philox4x32-10 (Salmon et al., SC 2011), from its published definition ----
struct U4 {
  uint32_t x, y, z, w;
};

__host__ __device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * c.x;
    uint64_t p1 = (uint64_t)M1 * c.z;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    U4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
  }
  return c;
}

// Entry `row` of random vector number `vec` of `stream`: exact value in [-1/2, 1/2).
__host__ __device__ inline double philox_pm_half(uint64_t seed, uint32_t stream, uint32_t vec,
                                                 uint32_t row) {
  U4 c{row, vec, stream, 0u};
  U4 r = philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  uint64_t u53 = ((uint64_t)(r.x >> 5) << 26) | (uint64_t)(r.y >> 6);
  return (double)u53 * 0x1.0p-53 - 0.5;
}

// Kernel launches issued by this library (all threads, all handles); read by
// bchdav_solve to report the launches of one solve.
extern unsigned long long g_launches;
inline void note_launch() { __atomic_fetch_add(&g_launches, 1ull, __ATOMIC_RELAXED); }

constexpr uint32_t kStreamReplace = 1;
constexpr uint32_t kStreamFill = 2;
constexpr uint32_t kStreamLanczos = 3;   // start vector of the Lanczos bound estimate

}  // namespace bchdav
