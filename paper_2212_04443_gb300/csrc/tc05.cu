// The slice products of csrc/ozaki.cu on the 5th-generation tensor cores (tcgen05.mma, operands
// in shared memory, float32 level sums in tensor memory):
//   MODE 0  C (n x nb)  = A B      Step 11 rotation V <- V Y (A: row planes of V)
//   MODE 1  C (n x nb) -= A B      Step 6 update X -= V C
//   MODE 2  out (ka x kb) = A^T B  Steps 6 and 8 Gram products V^T X, V^T W (A, B: transposed
//                                  column planes, the reduction over the N rows)
//
// Operands.  The digit planes are stored tiled (oz_tix in ozaki.cu): one 16-wide k step of a run
// of consecutive rows is, for each slice and each half of the step, 16 contiguous bytes per row.
// Viewed with 8-byte elements (a row's 16 bytes are two elements), a 128-row run of one slice
// and half is one 2 KB box row, so ONE TMA box per k step brings a 128-row tile of A for every
// slice and half (16 box rows), and two boxes bring B's 32-row tile (one per half of the step,
// every slice).  They land as no-swizzle K-major core matrices (8 rows x 16 bytes, 128 bytes
// apart in M or N; the two k halves of a slice a row block apart).  (16-byte box rows, one per
// row, would leave the TMA unit walking 2,560 rows per k step.)
//
// Products per k step: A's slice s against B's slices 0 .. S-1-s side by side (B's stage holds
// the slices' 32-row blocks one after another), one tcgen05.mma M128 x N32(S - s) x K16 into the
// level sums starting at block s: slice pair (s, t) lands in block s + t, its level.  S
// instructions per k step instead of S (S + 1) / 2.
//
// Level sums.  Level L = s + t has weight 2^(-6 (L + 2)).  A level sum is an integer below 2^23
// (at most 8 products of at most 1024 terms of digits bounded by 64 x 32, 64 x 64 only for the
// single pair of level 0), exact in float32.  They are folded EXACTLY in 64-bit integers,
// hi = sum_{L < H} acc_L 2^(6 (H - 1 - L)) and lo = sum_{L >= H} acc_L 2^(6 (S - 1 - L)) with
// H = S / 2 (each below 2^42), and converted to float64 once:
//   value = (hi 2^(6 (S - H)) + lo) 2^(-6 (S + 1)) 2^(E_row + F_col).
// The Gram products fold every 1024 rows (one exponent chunk) with that chunk's exponents.
//
// Warp roles in a persistent CTA of 192 threads (one per SM):
//   warp 0, one lane   producer: TMA boxes of each k step into a 4-stage ring (full/empty
//                      mbarriers);
//   warp 1, one lane   issuer: the S products of each k step; a tile's (or a Gram chunk's) level
//                      sums alternate between two tensor-memory buffers (2 x S x 32 columns), so
//                      the next tile's products overlap this one's fold;
//   warps 2-5          fold: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its 32 output
//                      rows), folds the level sums and writes C (MODE 0/1) or accumulates the
//                      Gram chunks in float64 registers and writes the unit's partial sums.
// Every wait is bounded; a role whose wait expires sets the CTA's failure flag, which makes the
// others stop at their next wait; before the shared and tensor memory are released the producer
// waits (bounded) for the copies it issued that no product consumed and the issuer for every
// product it issued.  The host reads the error flag (BCHDAV_ERR_TIMEOUT).
#include <algorithm>
#include <cstdlib>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "kernels.cuh"

namespace bchdav {
namespace {

constexpr int kTcM = 128;        // A tile rows (tensor-memory lanes)
constexpr int kTcN = 32;         // B tile rows (output columns per level block)
constexpr int kTcK = 16;         // k per instruction (kind::f16)
constexpr int kTcS = 8;          // digit slices stored per operand
constexpr int kTcStages = 4;
constexpr int kTcThreads = 192;
constexpr int kTcChunk = 64;     // k steps per exponent chunk of a Gram product (1024 rows)
constexpr long long kTcSpin = 1LL << 26;   // mbarrier polls before a wait is declared failed

template <int NS>
constexpr size_t tc_smem_bytes() {
  return (size_t)kTcStages * NS * 2 * (kTcM + kTcN) * 16 + 256;
}

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
// N = n (a multiple of 16, at most 256), M = 128
__host__ __device__ constexpr unsigned tc_idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) |
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

__device__ __forceinline__ bool mbar_try(unsigned mbar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait: gives up after `limit` polls, or early once another role set *fail
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity, volatile int* fail,
                                          long long limit = kTcSpin) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try(mbar, parity)) return true;
    if (fail && (i & 1023) == 1023 && *fail) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_expect(unsigned mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
               : "memory");
}

// TMA over the 8-byte element view of tiled planes (tc_map_runs): box at (2 row, 0, k block)
__device__ __forceinline__ void tma_runs(unsigned dst, const CUtensorMap* map, int row, int kb,
                                         unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3, %4}], [%5];\n" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(2 * row), "r"(0), "r"(kb), "r"(mbar)
      : "memory");
}
// ... and over its per-half view (tc_map_runs_half): box at (2 row, half, 0, k block)
__device__ __forceinline__ void tma_runs_half(unsigned dst, const CUtensorMap* map, int row,
                                              int half, int kb, unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3, %4, %5}], [%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(2 * row), "r"(half), "r"(0), "r"(kb),
      "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld8(unsigned (&r)[8], unsigned taddr) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
}

__device__ __forceinline__ double tc_pow2(int ex) {
  return (ex > -1022 && ex < 1023) ? __longlong_as_double((long long)(ex + 1023) << 52)
                                   : ldexp(1.0, ex);
}

struct TcWork {
  int mode_rows;     // MODE 0/1: output rows n; MODE 2: output rows ka
  int ncols;         // output columns (nb or kb)
  int nk;            // k steps
  int m_tiles, n_tiles, n_units;
  int chunks_per_unit;   // MODE 2
  int a_row0;        // MODE 2: first row of A's planes (column of V)
};

template <int MODE, int NS>
__global__ void __launch_bounds__(kTcThreads, 1) tc_slice_kernel(
    const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcWork wk,
    const int* __restrict__ EA, int strideA, const int* __restrict__ EB, int strideB,
    double* __restrict__ C, int ldc, int* __restrict__ err, int expire_first_wait) {
  constexpr int kAStage = NS * 2 * kTcM * 16;
  constexpr int kBStage = NS * 2 * kTcN * 16;
  constexpr int kH = NS / 2;
  constexpr int kCols = 2 * NS * kTcN <= 256 ? 256 : 512;   // tensor-memory columns
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* sA = tc_smem;
  unsigned char* sB = tc_smem + (size_t)kTcStages * kAStage;
  unsigned long long* full = reinterpret_cast<unsigned long long*>(sB + (size_t)kTcStages * kBStage);
  unsigned long long* empty = full + kTcStages;
  unsigned long long* tfull = empty + kTcStages;   // 2 buffers
  unsigned long long* tempty = tfull + 2;          // 2 buffers
  unsigned long long* done = tempty + 2;
  unsigned long long* never = done + 1;            // nothing arrives on it (timeout test)
  unsigned* tslot = reinterpret_cast<unsigned*>(never + 1);
  volatile int* s_fail = reinterpret_cast<volatile int*>(tslot + 1);
  long long* s_count = reinterpret_cast<long long*>(tslot + 2);   // [0] issued, [1] consumed

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nk = wk.nk;
  const int nch = MODE == 2 ? (nk + kTcChunk - 1) / kTcChunk : 1;
  if (t == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(full + i)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(empty + i)));
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(tfull + i)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(smem_u32(tempty + i)));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(done)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(never)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *s_fail = 0;
    s_count[0] = 0;
    s_count[1] = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tslot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = *tslot;

  // unit u.  MODE 0/1: (row tile, column tile), column tiles of a row tile adjacent (they share
  // A's tile in L2); every k step, one fold.  MODE 2: (A tile, B tile, range of whole chunks).
  auto unit = [&](int u, int& mt, int& nt, int& c0, int& c1) {
    if (MODE == 2) {
      mt = u % wk.m_tiles;
      const int rem = u / wk.m_tiles;
      nt = rem % wk.n_tiles;
      c0 = (rem / wk.n_tiles) * wk.chunks_per_unit;
      c1 = min(nch, c0 + wk.chunks_per_unit);
    } else {
      mt = u / wk.n_tiles;
      nt = u - mt * wk.n_tiles;
      c0 = 0;
      c1 = 1;
    }
  };
  auto ks_range = [&](int ch, int& k0, int& k1) {
    k0 = MODE == 2 ? ch * kTcChunk : 0;
    k1 = MODE == 2 ? min(nk, (ch + 1) * kTcChunk) : nk;
  };
  const int a_row0 = MODE == 2 ? wk.a_row0 : 0;

  if (warp == 0) {
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < wk.n_units && ok; u += gridDim.x) {
        int mt, nt, c0, c1;
        unit(u, mt, nt, c0, c1);
        for (int ch = c0; ch < c1 && ok; ++ch) {
          int k0, k1;
          ks_range(ch, k0, k1);
          for (int ks = k0; ks < k1; ++ks) {
            const int st = (int)(it % kTcStages);
            if (it >= kTcStages &&
                !mbar_wait(smem_u32(empty + st), (unsigned)(((it / kTcStages) - 1) & 1), s_fail)) {
              ok = false;
              break;
            }
            const unsigned fb = smem_u32(full + st);
            mbar_expect(fb, (unsigned)(kAStage + kBStage));
            const unsigned b0 = smem_u32(sB + (size_t)st * kBStage);
            tma_runs(smem_u32(sA + (size_t)st * kAStage), &mapA, a_row0 + mt * kTcM, ks, fb);
            tma_runs_half(b0, &mapB, nt * kTcN, 0, ks, fb);
            tma_runs_half(b0 + (unsigned)(NS * kTcN * 16), &mapB, nt * kTcN, 1, ks, fb);
            ++it;
            s_count[0] = it;
          }
        }
      }
      if (!ok) *s_fail = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long it = 0, f = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < wk.n_units && ok; u += gridDim.x) {
        int mt, nt, c0, c1;
        unit(u, mt, nt, c0, c1);
        for (int ch = c0; ch < c1 && ok; ++ch) {
          const int buf = (int)(f & 1);
          if (f >= 2 &&
              !mbar_wait(smem_u32(tempty + buf), (unsigned)(((f >> 1) - 1) & 1), s_fail)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const unsigned dbase = tmem + (unsigned)(buf * NS * kTcN);
          int k0, k1;
          ks_range(ch, k0, k1);
          for (int ks = k0; ks < k1; ++ks) {
            const int st = (int)(it % kTcStages);
            // expire_first_wait (tests of the timeout path only): the first wait polls a
            // barrier nothing arrives on, briefly
            if (expire_first_wait && it == 0 && !mbar_wait(smem_u32(never), 0, nullptr, 1000)) {
              ok = false;
              break;
            }
            if (!mbar_wait(smem_u32(full + st), (unsigned)((it / kTcStages) & 1), s_fail)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // A stage [slice][half][128 rows][16 B]: slice s at s x 4 KB, its k halves 2 KB apart.
            // B stage [half][slice][32 rows][16 B]: slices 0 .. NS-1-s are one operand of
            // 32 (NS - s) rows, its k halves NS x 512 B apart.
            const unsigned long long da =
                tc_desc(smem_u32(sA + (size_t)st * kAStage), kTcM * 16, 128);
            const unsigned long long db =
                tc_desc(smem_u32(sB + (size_t)st * kBStage), NS * kTcN * 16, 128);
#pragma unroll
            for (int s2 = 0; s2 < NS; ++s2)
              tc_mma(dbase + (unsigned)(s2 * kTcN),
                     da + (unsigned long long)((s2 * 2 * kTcM * 16) >> 4), db,
                     tc_idesc_n(kTcN * (NS - s2)), (ks > k0 || s2 > 0) ? 1 : 0);
            tc_commit(smem_u32(empty + st));
            ++it;
            s_count[1] = it;
          }
          if (!ok) break;
          tc_commit(smem_u32(tfull + buf));
          ++f;
        }
      }
      if (!ok) *s_fail = 1;
      // every product issued must finish before the tensor memory goes away
      tc_commit(smem_u32(done));
      if (!mbar_wait(smem_u32(done), 0, nullptr)) *s_fail = 1;
    }
  } else {
    // fold warps: tensor-memory lanes 32 (warp % 4) .. + 31
    const int q = warp & 3;
    const bool small_k = MODE != 2 && nk <= 2;
    long long f = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < wk.n_units && ok; u += gridDim.x) {
      int mt, nt, c0, c1;
      unit(u, mt, nt, c0, c1);
      const int row = mt * kTcM + q * 32 + lane;   // output row (MODE 2: column of V, local)
      const bool row_ok = row < wk.mode_rows;
      const int Erow = (MODE != 2 && row_ok) ? EA[row] : 0;
      double acc[kTcN];
#pragma unroll
      for (int j = 0; j < kTcN; ++j) acc[j] = 0.0;
      for (int ch = c0; ch < c1; ++ch) {
        const int buf = (int)(f & 1);
        if (!mbar_wait(smem_u32(tfull + buf), (unsigned)((f >> 1) & 1), s_fail)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int Ea = MODE == 2 ? (row_ok ? EA[(size_t)ch * strideA + row] : 0) : Erow;
        const unsigned tbase = tmem + ((unsigned)(q * 32) << 16) + (unsigned)(buf * NS * kTcN);
#pragma unroll
        for (int g = 0; g < kTcN / 8; ++g) {
          if (nt * kTcN + g * 8 >= wk.ncols) break;   // no output column left in this tile
          unsigned r[NS][8];
#pragma unroll
          for (int L = 0; L < NS; ++L) tmem_ld8(r[L], tbase + (unsigned)(L * kTcN + g * 8));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            long long hi = 0, lo = 0;
#pragma unroll
            for (int L = 0; L < NS; ++L) {
              const long long v = (long long)__float2int_rn(__uint_as_float(r[L][i]));
              if (L < kH) hi += v * (1LL << (6 * (kH - 1 - L)));
              else lo += v * (1LL << (6 * (NS - 1 - L)));
            }
            const int col = nt * kTcN + g * 8 + i;
            if (col < wk.ncols && row_ok) {
              // K <= 32 (one or two k steps): every level sum is below 2^20, so the whole
              // integer fits in 64 bits and one conversion suffices
              const double v =
                  small_k ? (double)(hi * (1LL << (6 * (NS - kH))) + lo)
                          : fma((double)hi, (double)(1LL << (6 * (NS - kH))), (double)lo);
              const int Eb = MODE == 2 ? EB[(size_t)ch * strideB + col] : EB[col];
              acc[g * 8 + i] = fma(v, tc_pow2(Ea + Eb - 6 * (NS + 1)), acc[g * 8 + i]);
            }
          }
        }
        // the buffer may be overwritten once every fold warp has read it
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(tempty + buf))
                       : "memory");
        ++f;
      }
      if (!ok) break;
      if (row_ok) {
        if (MODE == 2) {
          const int sp = u / (wk.m_tiles * wk.n_tiles);
          double* out = C + ((size_t)sp * wk.mode_rows + row) * wk.ncols;
#pragma unroll
          for (int j = 0; j < kTcN; ++j) {
            const int col = nt * kTcN + j;
            if (col < wk.ncols) out[col] = acc[j];
          }
        } else {
          double* out = C + (size_t)row * ldc;
#pragma unroll
          for (int j = 0; j < kTcN; ++j) {
            const int col = nt * kTcN + j;
            if (col < wk.ncols) {
              if (MODE == 0) out[col] = acc[j];
              else out[col] -= acc[j];
            }
          }
        }
      }
    }
    if (!ok) *s_fail = 1;
  }
  __syncthreads();
  if (t == 0) {
    // copies issued that no product consumed (after a failure) must land before shared memory
    // is released
    const long long issued = s_count[0], consumed = s_count[1];
    for (long long p = consumed; p < issued; ++p)
      if (!mbar_wait(smem_u32(full + (int)(p % kTcStages)), (unsigned)((p / kTcStages) & 1),
                     nullptr))
        *s_fail = 1;
    if (*s_fail) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 1)
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

// Tiled planes (oz_tix: `cap` rows, Kp values of k) viewed with 8-byte elements: 3-d tensor
// (2 rows, 16 slice halves, Kp / 16 k blocks); rows at or past `rows` read as zeros.  Box
// (2 box_rows, 2 slices, 1): every slice and half of one k step of box_rows rows, landing as
// [slice][half][rows][16 bytes]; each box row is 16 box_rows contiguous bytes.
bool tc_map_runs(CUtensorMap* m, const void* planes, int rows, int cap, int Kp, int box_rows,
                 int slices) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc_encoder();
  if (!enc || rows < 1 || rows > cap || Kp % kTcK != 0 || 2 * box_rows > 256) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)rows * 2, (cuuint64_t)(2 * kTcS), (cuuint64_t)(Kp / kTcK)};
  const cuuint64_t strides[2] = {(cuuint64_t)cap * 16, (cuuint64_t)cap * 16 * 2 * kTcS};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * box_rows), (cuuint32_t)(2 * slices), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(planes), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The same view as a 4-d tensor (2 rows, 2 halves, 8 slices, k blocks); box (2 box_rows, 1,
// slices, 1): one half of a k step for every slice, landing as [slice][rows][16 bytes]
bool tc_map_runs_half(CUtensorMap* m, const void* planes, int rows, int cap, int Kp, int box_rows,
                      int slices) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc_encoder();
  if (!enc || rows < 1 || rows > cap || Kp % kTcK != 0 || 2 * box_rows > 256) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)rows * 2, 2, (cuuint64_t)kTcS, (cuuint64_t)(Kp / kTcK)};
  const cuuint64_t strides[3] = {(cuuint64_t)cap * 16, (cuuint64_t)cap * 32,
                                 (cuuint64_t)cap * 16 * 2 * kTcS};
  const cuuint32_t box[4] = {(cuuint32_t)(2 * box_rows), 1, (cuuint32_t)slices, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void*>(planes), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int tc_sms() {
  static const int sms = []() {
    int dev = 0, v = kSMs;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : kSMs;
  }();
  return sms;
}

template <int MODE, int NS>
cudaError_t tc_run(cudaStream_t st, const CUtensorMap& mA, const CUtensorMap& mB, const TcWork& wk,
                   const int* EA, int strideA, const int* EB, int strideB, double* C, int ldc,
                   int* err) {
  static const cudaError_t attr = cudaFuncSetAttribute(
      tc_slice_kernel<MODE, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)tc_smem_bytes<NS>());
  if (attr != cudaSuccess) return attr;
  const int grid = std::min(wk.n_units, tc_sms());
  if (grid <= 0) return cudaSuccess;
  // BCHDAV_TEST_EXPIRE_TC_WAIT=1 (tests of the timeout path only): see expire_first_wait
  const char* env = getenv("BCHDAV_TEST_EXPIRE_TC_WAIT");
  const int expire = env && env[0] == '1' ? 1 : 0;
  tc_slice_kernel<MODE, NS><<<grid, kTcThreads, tc_smem_bytes<NS>(), st>>>(
      mA, mB, wk, EA, strideA, EB, strideB, C, ldc, err, expire);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

// C (n x nb) = / -= A B: A's row planes (tiled, n rows, Kp values of k, row exponents EA), B's
// column planes (tiled, nbp >= nb rows, column exponents EB), the leading `slices` digit planes
// (8; 6 for a product C = A B whose operands may keep 36 bits).  err: set when a wait expired.
cudaError_t launch_tc_slice_nn(cudaStream_t st, int n, int nb, int Kp, const void* PA,
                               const int* EA, const void* PB, int nbp, const int* EB, double* C,
                               int ldc, bool subtract, int slices, int* err) {
  if (n <= 0 || nb <= 0 || Kp <= 0) return cudaSuccess;
  if (Kp % kTcK != 0 || nb > nbp || Kp > 448 + kTcK) return cudaErrorInvalidValue;
  if (subtract && slices != 8) return cudaErrorInvalidValue;
  if (slices != 8 && slices != 6) return cudaErrorInvalidValue;
  CUtensorMap mA, mB;
  if (!tc_map_runs(&mA, PA, n, n, Kp, kTcM, slices) ||
      !tc_map_runs_half(&mB, PB, nb, nbp, Kp, kTcN, slices))
    return cudaErrorInvalidValue;
  TcWork wk;
  wk.mode_rows = n;
  wk.ncols = nb;
  wk.nk = Kp / kTcK;
  wk.m_tiles = ceil_div(n, kTcM);
  wk.n_tiles = ceil_div(nb, kTcN);
  wk.n_units = wk.m_tiles * wk.n_tiles;
  wk.chunks_per_unit = 1;
  wk.a_row0 = 0;
  if (subtract) return tc_run<1, 8>(st, mA, mB, wk, EA, 0, EB, 0, C, ldc, err);
  if (slices == 6) return tc_run<0, 6>(st, mA, mB, wk, EA, 0, EB, 0, C, ldc, err);
  return tc_run<0, 8>(st, mA, mB, wk, EA, 0, EB, 0, C, ldc, err);
}

// out (ka x kb) = A^T B from the transposed column planes (see oz_gram_from_planes): rows
// [a0, a0 + ka) of PA (tiled, capA rows, Np values of k, chunk exponents EA with stride capA)
// and rows [0, kb) of PB (tiled, capB rows, chunk exponents EB, stride capB); the leading
// `slices` digit planes of both.  partial: room for (number of SMs) x ka x kb doubles.  err: set
// when a wait expired.
cudaError_t launch_tc_gram(cudaStream_t st, int Np, const void* PA, const int* EA, int capA, int a0,
                           int ka, const void* PB, const int* EB, int capB, int kb, double* out,
                           double* partial, int slices, int* err) {
  if (ka <= 0 || kb <= 0) return cudaSuccess;
  if (Np % kTcK != 0 || a0 < 0 || a0 + ka > capA || kb > capB) return cudaErrorInvalidValue;
  CUtensorMap mA, mB;
  if ((slices != 8 && slices != 6 && slices != 4) ||
      !tc_map_runs(&mA, PA, a0 + ka, capA, Np, kTcM, slices) ||
      !tc_map_runs_half(&mB, PB, kb, capB, Np, kTcN, slices))
    return cudaErrorInvalidValue;
  TcWork wk;
  wk.mode_rows = ka;
  wk.ncols = kb;
  wk.nk = Np / kTcK;
  wk.m_tiles = ceil_div(ka, kTcM);
  wk.n_tiles = ceil_div(kb, kTcN);
  const int nch = ceil_div(wk.nk, kTcChunk);
  const int tiles = wk.m_tiles * wk.n_tiles;
  int splits = std::max(1, std::min(nch, tc_sms() / tiles));
  wk.chunks_per_unit = ceil_div(nch, splits);
  splits = ceil_div(nch, wk.chunks_per_unit);
  wk.n_units = tiles * splits;
  wk.a_row0 = a0;
  const int* ea = EA + a0;
  cudaError_t e;
  if (slices == 8) e = tc_run<2, 8>(st, mA, mB, wk, ea, capA, EB, capB, partial, 0, err);
  else if (slices == 6) e = tc_run<2, 6>(st, mA, mB, wk, ea, capA, EB, capB, partial, 0, err);
  else e = tc_run<2, 4>(st, mA, mB, wk, ea, capA, EB, capB, partial, 0, err);
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(st, partial, splits, ka * kb, out, 1.0);
}

}  // namespace bchdav
