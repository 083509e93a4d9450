// The row-operand slice products C (n x nb) = / -= A B of csrc/ozaki.cu (Step 11 rotation,
// Step 6 update X -= V C) on the 5th-generation tensor cores: tcgen05.mma with operands in
// shared memory (K-major 8x16-byte core matrices, no swizzle) and the float32 level sums in
// tensor memory (one BN-column region per level of a 128 x BN output tile, BN = 32 or 64).
//
// The digit planes, exponents and level weights are those of csrc/ozaki.cu: A's row planes
// (S x n x Kp, row exponents EA), B's column planes (S x nbp x Kp, column exponents EB);
// level L = s + t of slice pair (s, t) has weight 2^(-6 (L + 2)); each level sums at most 8
// products of K <= 448 terms of integers bounded by 64 * 64, exact in float32.
//
// One persistent CTA per SM walks its 128 x BN output tiles as one sequence of 16-wide k steps.
// Thread 0 is the producer and the tensor-core issuer: per step it waits for the step's
// operands (an mbarrier completed by the tensor-memory-access (TMA) copies), issues the
// tcgen05.mma of every slice pair, commits them to the stage's "empty" mbarrier, and issues the
// TMA copies of the step three ahead into the stage the previous step has finished with.  The
// copies are 3-d boxes (8 k x rows x 1 slice) of the digit planes; each box lands as rows of 16
// bytes, which is the no-swizzle K-major core-matrix layout (core matrices 128 bytes apart in
// M or N, the two k halves a box apart).  At a tile's end the four warps read the level sums
// from tensor memory, combine them in float64, scale by 2^(E_row + F_col) and write C.  Every
// wait on an mbarrier is bounded: on expiry the CTA records an error, stops issuing, and still
// waits (also bounded) for the copies and products it issued before it frees the tensor memory
// and returns.
#include <cstdlib>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "kernels.cuh"

namespace bchdav {
namespace {

constexpr int kTcM = 128;        // output rows per CTA (tensor-memory lanes)
constexpr int kTcK = 16;         // k per instruction (kind::f16)
constexpr int kTcS = 8;          // digit slices stored per operand
constexpr int kTcStages = 4;
constexpr int kTcThreads = 128;
constexpr long long kTcSpin = 1LL << 26;   // mbarrier polls before a wait is declared failed

constexpr int kTcAStage = kTcS * kTcM * kTcK * 2;   // 32 KB
constexpr int kTcBStage = kTcS * 64 * kTcK * 2;     // 16 KB (room for 64 output columns)
constexpr size_t kTcSmem = (size_t)kTcStages * (kTcAStage + kTcBStage) + 512;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major, no swizzle; lbo / sbo = byte distance between
// core matrices adjacent in K / in M (or N); bits 46-47 = 1 (descriptor version)
__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr >> 4) & 0x3FFF);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFF) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFF) << 32;
  d |= 1ull << 46;
  return d;
}

// instruction descriptor, kind::f16: float32 accumulator, bf16 A and B, both K-major,
// N = BN, M = 128
template <int BN>
__host__ __device__ constexpr unsigned tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(BN >> 3) << 17) |
         ((unsigned)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned dtmem, unsigned long long ad, unsigned long long bd,
                                       unsigned idesc, int accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity,
                                          long long limit = kTcSpin) {
  for (long long i = 0; i < limit; ++i) {
    unsigned done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mbar_expect(unsigned mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
               : "memory");
}

// TMA: box (8 k, rows, 1 slice) at coordinates (x = k, y = row, z = slice) into shared memory
__device__ __forceinline__ void tma_load3(unsigned dst, const CUtensorMap* map, int x, int y, int z,
                                          unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3, %4}], [%5];\n" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}

template <int MODE, int NS, int BN>
__global__ void __launch_bounds__(kTcThreads, 1) tc_slice_nn_kernel(
    const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int n,
    int nb, int Kp, const int* __restrict__ EA, const int* __restrict__ EB,
    double* __restrict__ C, int ldc, int* __restrict__ err, int expire_first_wait) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* sA = tc_smem;                                      // [stage][s][h] 2 KB each
  unsigned char* sB = tc_smem + (size_t)kTcStages * kTcAStage;      // [stage][s][h] BN x 16 B
  unsigned long long* full =
      reinterpret_cast<unsigned long long*>(sB + (size_t)kTcStages * kTcBStage);
  unsigned long long* empty = full + kTcStages;
  unsigned long long* tile_bar = empty + kTcStages;
  unsigned long long* never = tile_bar + 1;   // nothing arrives on it (error-path test)
  unsigned* tslot = reinterpret_cast<unsigned*>(never + 1);
  int* s_fail = reinterpret_cast<int*>(tslot + 1);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  constexpr int kCols = 8 * BN;   // tensor-memory columns allocated (a power of two >= 32)
  constexpr unsigned kStageBytes = NS * 2u * (kTcM + BN) * 16u;
  // tiles in order row-tile-major (the column tiles of one row tile are adjacent: they share
  // A's tile in L2); this CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...
  const int n_ct = (nb + BN - 1) / BN;
  const long long n_tiles = (long long)n_ct * ((n + kTcM - 1) / kTcM);
  const int my_tiles =
      blockIdx.x < n_tiles ? (int)((n_tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  const int nk = Kp / kTcK;
  const long long total = (long long)my_tiles * nk;   // (tile, k step) pairs of this CTA

  if (t == 0) {
    for (int i = 0; i < 2 * kTcStages + 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(full + i)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tslot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = *tslot;

  auto origin = [&](long long step, int& r0, int& c0, int& kt) {
    const long long j = step / nk;
    kt = (int)(step - j * nk);
    const long long tile = blockIdx.x + j * gridDim.x;
    c0 = (int)(tile % n_ct) * BN;
    r0 = (int)(tile / n_ct) * kTcM;
  };
  // thread 0's step cursors (no divisions on the issue path): the producer's next step and the
  // tile it lies in
  int pk = 0, pr0 = 0, pc0 = 0;
  long long ptile = blockIdx.x;
  auto advance = [&](int& k, long long& tile, int& r0, int& c0) {
    if (++k == nk) {
      k = 0;
      tile += gridDim.x;
      c0 += (int)gridDim.x % n_ct * BN;   // tile advances by gridDim.x: carry into rows
      r0 += (int)(gridDim.x / n_ct) * kTcM;
      if (c0 >= n_ct * BN) {
        c0 -= n_ct * BN;
        r0 += kTcM;
      }
    }
  };
  {
    int k0;
    origin(0, pr0, pc0, k0);
  }
  // descriptor bases per stage (the slice offsets are added to the address field)
  unsigned long long dA[kTcStages], dB[kTcStages];
#pragma unroll
  for (int i = 0; i < kTcStages; ++i) {
    dA[i] = tc_desc(smem_u32(sA + (size_t)i * kTcAStage), kTcM * 16, 128);
    dB[i] = tc_desc(smem_u32(sB + (size_t)i * kTcBStage), BN * 16, 128);
  }
  // thread 0 only: copies of step p into stage p % kTcStages
  long long issued = 0, consumed = 0;
  unsigned bar_commits = 0;   // commits on tile_bar so far
  bool fail = false;
  auto produce = [&](long long p) {
    const int st = (int)(p % kTcStages);
    if (p >= kTcStages &&
        !mbar_wait(smem_u32(empty + st), (unsigned)(((p / kTcStages) - 1) & 1))) {
      fail = true;
      return;
    }
    const int r0 = pr0, c0 = pc0, kt = pk;
    advance(pk, ptile, pr0, pc0);
    const unsigned fb = smem_u32(full + st);
    mbar_expect(fb, kStageBytes);
    const unsigned a0 = smem_u32(sA + (size_t)st * kTcAStage);
    const unsigned b0 = smem_u32(sB + (size_t)st * kTcBStage);
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        tma_load3(a0 + (unsigned)(s * 2 + h) * (kTcM * 16), &mapA, kt * kTcK + h * 8, r0, s, fb);
        tma_load3(b0 + (unsigned)(s * 2 + h) * (BN * 16), &mapB, kt * kTcK + h * 8, c0, s, fb);
      }
    issued = p + 1;
  };
  auto consume = [&](long long g, int kt) {
    const int st = (int)(g % kTcStages);
    // expire_first_wait (tests only): the first wait polls a barrier nothing arrives on, briefly,
    // so that the error path below runs without any fault
    if (expire_first_wait && g == 0 && !mbar_wait(smem_u32(never), 0, 1000)) {
      fail = true;
      return;
    }
    if (!mbar_wait(smem_u32(full + st), (unsigned)((g / kTcStages) & 1))) {
      fail = true;
      return;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      // A slice s: core matrices 128 B apart along M, the k halves 2 KB apart (the address
      // field of the descriptor counts 16-byte units)
      const unsigned long long ad = dA[st] + (unsigned long long)((s * 2 * kTcM * 16) >> 4);
#pragma unroll
      for (int u = 0; u < NS; ++u) {
        if (s + u < NS) {
          const unsigned long long bd = dB[st] + (unsigned long long)((u * 2 * BN * 16) >> 4);
          // level s + u starts fresh at a tile's first k step with its first pair (0, level)
          tc_mma(tmem + (unsigned)((s + u) * BN), ad, bd, tc_idesc<BN>(), (kt > 0 || s > 0) ? 1 : 0);
        }
      }
    }
    tc_commit(smem_u32(empty + st));
    consumed = g + 1;
  };

  for (int j = 0; j < my_tiles; ++j) {
    if (t == 0) {
      if (j == 0)
        for (long long p = 0; p < kTcStages - 1 && p < total && !fail; ++p) produce(p);
      for (int kt = 0; kt < nk && !fail; ++kt) {
        const long long g = (long long)j * nk + kt;
        consume(g, kt);
        if (!fail && g + kTcStages - 1 < total) produce(g + kTcStages - 1);
      }
      if (fail) *s_fail = 1;
      tc_commit(smem_u32(tile_bar));   // completes once every product issued so far has
    }
    ++bar_commits;   // every thread counts the commit thread 0 made
    __syncwarp();
    bool ok = mbar_wait(smem_u32(tile_bar), (bar_commits - 1) & 1);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!ok) atomicExch(s_fail, 1);
    __syncthreads();
    if (*s_fail) break;
    int r0, c0, kt;
    origin((long long)j * nk, r0, c0, kt);
    // epilogue: warp w owns tensor-memory lanes (rows) 32w .. 32w + 31
    const int row = r0 + warp * 32 + lane;
    const int Er = row < n ? EA[row] : 0;
#pragma unroll 1
    for (int cc = 0; cc < BN / 16; ++cc) {
      double v[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) v[c] = 0.0;
#pragma unroll
      for (int L = NS - 1; L >= 0; --L) {
        unsigned r[16];
        const unsigned ta = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(L * BN + cc * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
            "%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
              "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        const double w = __longlong_as_double((long long)(1023 - 6 * (L + 2)) << 52);
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = fma((double)__uint_as_float(r[c]), w, v[c]);
      }
      if (row < n) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int col = c0 + cc * 16 + c;
          if (col >= nb) continue;
          const int ex = Er + EB[col];
          const double scale = (ex > -1022 && ex < 1023)
                                   ? __longlong_as_double((long long)(ex + 1023) << 52)
                                   : ldexp(1.0, ex);
          if (MODE == 0) C[(size_t)row * ldc + col] = v[c] * scale;
          else C[(size_t)row * ldc + col] -= v[c] * scale;
        }
      }
    }
    // the next tile's first products overwrite tensor memory only after every read above
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
  }
  if (t == 0) {
    // copies issued but not consumed (a failure), then every product: all must land before
    // the shared and tensor memory go away
    for (long long p = consumed; p < issued; ++p)
      if (!mbar_wait(smem_u32(full + (int)(p % kTcStages)), (unsigned)((p / kTcStages) & 1)))
        *s_fail = 1;
    tc_commit(smem_u32(tile_bar));
    if (!mbar_wait(smem_u32(tile_bar), bar_commits & 1)) *s_fail = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (*s_fail && t == 0) atomicExch(err, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kCols));
}

PFN_cuTensorMapEncodeTiled_v12000 tc_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// planes S x rows x Kp (bf16, k contiguous) as a 3-d tensor (Kp, rows, 8), boxes 8 x box_rows x 1
bool tc_map(CUtensorMap* m, const void* planes, int rows, int Kp, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)kTcS};
  const cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
  const cuuint32_t box[3] = {8, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(planes), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE, int NS, int BN>
cudaError_t tc_launch(cudaStream_t st, int n, int nb, int Kp, const void* PA, const int* EA,
                      const void* PB, int nbp, const int* EB, double* C, int ldc, int* err) {
  static const cudaError_t attr = cudaFuncSetAttribute(
      tc_slice_nn_kernel<MODE, NS, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (attr != cudaSuccess) return attr;
  CUtensorMap mA, mB;
  if (!tc_map(&mA, PA, n, Kp, kTcM) || !tc_map(&mB, PB, nbp, Kp, BN)) return cudaErrorInvalidValue;
  // persistent: one CTA per SM (the shared memory of the four stages admits one)
  const long long tiles = (long long)ceil_div(nb, BN) * ceil_div(n, kTcM);
  static const int sms = []() {
    int dev = 0, v = kSMs;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : kSMs;
  }();
  dim3 grid((unsigned)(tiles < sms ? tiles : sms));
  // BCHDAV_TEST_EXPIRE_TC_WAIT=1 (tests of the timeout path only): see expire_first_wait
  const char* env = getenv("BCHDAV_TEST_EXPIRE_TC_WAIT");
  const int expire = env && env[0] == '1' ? 1 : 0;
  tc_slice_nn_kernel<MODE, NS, BN><<<grid, kTcThreads, kTcSmem, st>>>(mA, mB, n, nb, Kp, EA, EB, C,
                                                                      ldc, err, expire);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

// B's planes must cover whole tiles: nbp a multiple of 32 (nb <= 32) or of 64.
cudaError_t launch_tc_slice_nn(cudaStream_t st, int n, int nb, int Kp, const void* PA,
                               const int* EA, const void* PB, int nbp, const int* EB, double* C,
                               int ldc, bool subtract, int slices, int* err) {
  if (n <= 0 || nb <= 0 || Kp <= 0) return cudaSuccess;
  if (Kp % kTcK != 0 || nb > nbp || Kp > 448 + kTcK) return cudaErrorInvalidValue;
  const bool narrow = nb <= 32;
  if (narrow ? nbp < 32 : nbp % 64 != 0) return cudaErrorInvalidValue;
  if (subtract) {
    if (slices != 8) return cudaErrorInvalidValue;
    return narrow ? tc_launch<1, 8, 32>(st, n, nb, Kp, PA, EA, PB, nbp, EB, C, ldc, err)
                  : tc_launch<1, 8, 64>(st, n, nb, Kp, PA, EA, PB, nbp, EB, C, ldc, err);
  }
  if (slices == 6)
    return narrow ? tc_launch<0, 6, 32>(st, n, nb, Kp, PA, EA, PB, nbp, EB, C, ldc, err)
                  : tc_launch<0, 6, 64>(st, n, nb, Kp, PA, EA, PB, nbp, EB, C, ldc, err);
  if (slices == 8)
    return narrow ? tc_launch<0, 8, 32>(st, n, nb, Kp, PA, EA, PB, nbp, EB, C, ldc, err)
                  : tc_launch<0, 8, 64>(st, n, nb, Kp, PA, EA, PB, nbp, EB, C, ldc, err);
  return cudaErrorInvalidValue;
}

}  // namespace bchdav
