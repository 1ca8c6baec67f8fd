// Bottleneck contraction (Sec. 4.2.9, Eq. BottleneckPart) on the 5th-generation
// tensor cores:
//   C[(c, n^), (n', n~)] = sum_{(rho, n^')} T[(c, n^), (rho, n^')] B[(n', n~), (rho, n^')]
// with both operands split into BF16 pieces, x = x_0 + x_1 (+ x_2), or into TF32
// pieces (FP32 words whose low 13 mantissa bits are zero), x = x_0 (+ x_1), and the
// product formed as a sum of piece products (terms) x_i y_j.
//
// Two persistent kernels; launch_tc_gemm uses the CTA-pair one (HOTRG_TC_USE_PAIR).
//
// tc_gemm_pair_kernel (cta_group::2): a cluster of two CTAs on two SMs computes a
// 256 x 256 tile of C; CTA 0 issues tcgen05.mma with M = 256, N = 256, K = 16.  CTA r
// holds rows 128 r .. of the A tile and rows 128 r .. of the B tile, so each SM
// receives only half of the B tile: the per-SM copy rate, not the tensor pipe or the
// L2, is what bounds the one-CTA form below.  K slabs of 128-byte rows (64 BF16 or 32
// TF32, 128-byte swizzle), every piece of a slab in one ring stage (6 / npieces stages
// of npieces x 32 KiB);
// kind::f16 MMAs take K = 16 BF16, kind::tf32 MMAs K = 8 TF32: 32 bytes of a row
// either way.  The TF32 pieces run only in this form.
//
// tc_gemm_kernel (cta_group::1): one CTA per SM walks 128 x 256 tiles; K slabs of 32
// BF16 (64-byte rows) in a 3-stage ring, every piece of a slab in one stage.
//
// In both, the CTAs walk the tiles (tile index blockIdx.x, + gridDim.x, ...; row
// tiles fastest, so the CTAs running at one time share the B tiles in L2); one lane of
// one warp streams the slabs with TMA, one lane of another issues the MMAs (BF16 x
// BF16 -> FP32) and releases ring slots with tcgen05.commit.  The tensor core's FP32
// accumulation truncates, so a long accumulation drifts towards zero: the K range is
// therefore cut into chunks of 64, each accumulated from zero in one of two TMEM
// buffers (used alternately) while eight epilogue warps drain the other buffer with
// tcgen05.ld (warp w owns TMEM lanes 32(w%4)..) and add the chunk into FP32 registers
// with round-to-nearest.  Within a chunk the small terms (order 2^-16, then 2^-8) go
// first, the leading term x_0 y_0 last: the small terms then truncate at their own
// (small) scale and only the four leading MMAs truncate at the scale of the result.
// Every mbarrier wait is bounded in time; an expired wait sets a global error flag
// that also makes the other CTAs give up.
#include <cuda.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <atomic>

#include "hotrg_internal.cuh"
#include "../../include/hotrg.h"

namespace hotrg {

namespace {
// Tile TM x TN of C per CTA; K slabs of TK BF16 (TK = 64: 128-byte rows with the
// 128-byte swizzle; TK = 32: 64-byte rows with the 64-byte swizzle); a ring of STAGES
// stages, each holding every piece of one slab of A and B.
#ifndef HOTRG_TC_TN
#define HOTRG_TC_TN 256
#endif
#ifndef HOTRG_TC_TK
#define HOTRG_TC_TK 32
#endif
#ifndef HOTRG_TC_STAGES
#define HOTRG_TC_STAGES 3
#endif
constexpr int TM = 128, TN = HOTRG_TC_TN, TK = HOTRG_TC_TK, STAGES = HOTRG_TC_STAGES, MAXP = 3;
static_assert(TK == 32 || TK == 64, "K slab of 32 or 64 BF16");
static_assert(TN == 128 || TN == 256, "N tile of 128 or 256");
constexpr int A_PIECE = TM * TK * 2;
constexpr int B_PIECE = TN * TK * 2;
constexpr int STAGE_BYTES = MAXP * (A_PIECE + B_PIECE);
constexpr int TMEM_COLS = 2 * TN;      // two TN-column FP32 accumulators
constexpr int SW_BYTES = TK * 2;       // swizzle width = row length in bytes
// Epilogue warps: EPI_WARPS / 4 per TMEM lane quarter, each draining EPI_COLS columns
#ifndef HOTRG_TC_EPI_WARPS
#define HOTRG_TC_EPI_WARPS 8
#endif
constexpr int EPI_WARPS = HOTRG_TC_EPI_WARPS;
static_assert(EPI_WARPS == 8 || EPI_WARPS == 16, "8 or 16 epilogue warps");
constexpr int EPI_COLS = TN / (EPI_WARPS / 4);      // 128 or 64
constexpr int LD_COLS = EPI_WARPS == 8 ? 32 : 16;   // columns per tcgen05.ld
constexpr int W_PROD = EPI_WARPS, W_MMA = EPI_WARPS + 1;
constexpr int NTHREADS = 32 * (EPI_WARPS + 2);      // epilogue warps + producer + MMA
constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + 256;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory of one CTA");
constexpr unsigned long long WAIT_NS = 4000000000ull;  // 4 s per wait
}  // namespace

// K slabs per accumulation chunk (chunk length TK x this along K; 64 by default)
#ifndef HOTRG_TC_CHUNK_SLABS
#define HOTRG_TC_CHUNK_SLABS (64 / HOTRG_TC_TK)
#endif
constexpr int CHUNK_SLABS = HOTRG_TC_CHUNK_SLABS;
static_assert(CHUNK_SLABS >= 1 && CHUNK_SLABS < STAGES, "a chunk must leave a ring stage to prefetch into");

struct TcTerms {
  int nterms;
  int nsmall;    // terms [0, nsmall) are of order 2^-8 or smaller, the rest leading
  int npieces;   // pieces of each operand loaded per K slab
  // term t: A piece (code >> 4t) & 3, B piece (code >> (4t + 2)) & 3 (kept in a
  // register: an indexed array would live in local memory on the MMA issuer's path)
  unsigned long long code;
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after WAIT_NS, or as soon as another thread of the
// CTA or another CTA has given up.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* cta_abort,
                          volatile int* g_err) {
  unsigned long long t0 = 0;
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 127u) == 0) {
      if (*cta_abort || *g_err) return false;
      unsigned long long t = gtimer();
      if (t0 == 0) t0 = t;
      else if (t - t0 > WAIT_NS) {
        *cta_abort = 1;
        atomicExch((int*)g_err, HOTRG_ETIMEOUT);
        return false;
      }
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(const CUtensorMap* map, void* dst, uint64_t* bar, int x,
                                            int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(su32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
      : "memory");
}

// Shared-memory matrix descriptor for a K-major operand tile written by TMA with
// the SW_BYTES swizzle: rows of SW_BYTES bytes (TK BF16 along K), 8-row groups
// 8 SW_BYTES apart (the swizzle pattern repeats every 8 rows).
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);         // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused for this layout)
  d |= (uint64_t)((8 * SW_BYTES) >> 4) << 32;       // stride byte offset: 8 rows
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)(SW_BYTES == 128 ? 2 : 4) << 61;   // 128- or 64-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, N, M.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32 (format 2), both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32_f32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 lanes x 32 (or 16) columns of FP32 from TMEM; usable after tmem_wait_ld()
__device__ __forceinline__ void tmem_ld_async(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_async(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   float* __restrict__ C, int M, int N, long long ldc, int kslabs, TcTerms terms,
                   int* g_err) {
  extern __shared__ uint8_t smem_raw[];
  volatile int* gerr = g_err;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;      // [2] MMA -> epilogue
  uint64_t* tempty = tfull + 2;          // [2] epilogue -> MMA
  uint64_t* drain = tempty + 2;          // MMA completion on the abort path
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* cta_abort = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mtiles = (M + TM - 1) / TM;
  const long long ntiles = (long long)mtiles * ((N + TN - 1) / TN);
  // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...; one chunk per K slab
  const long long tiles_here =
      ntiles > (long long)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int np = terms.npieces;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, EPI_WARPS);
    }
    mbar_init(drain, 1);
    *cta_abort = *gerr ? 1 : 0;   // an earlier launch or CTA gave up: do nothing
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmB) : "memory");
  }
  if (warp == W_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // read once, after the barrier, so that every thread of the CTA takes the same path
  const long long my_tiles = *cta_abort ? 0 : tiles_here;
  const long long total = my_tiles * kslabs;

  if (warp == W_PROD) {
    if (lane == 0) {
      // ---------------- TMA producer: slab g of this CTA = K slab g % kslabs of
      // tile blockIdx.x + (g / kslabs) * gridDim.x; all pieces of A and B
      long long issued = 0;
      bool ok = true;
      for (long long g = 0; g < total; ++g) {
        const int s = (int)(g % STAGES);
        const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
        if (!mbar_wait(empty + s, ph ^ 1u, cta_abort, gerr)) {
          ok = false;
          break;
        }
        const long long tile = blockIdx.x + (g / kslabs) * gridDim.x;
        const int kb = (int)(g % kslabs);
        const int m0 = (int)(tile % mtiles) * TM, n0 = (int)(tile / mtiles) * TN;
        uint8_t* st = smem + s * STAGE_BYTES;
        mbar_expect_tx(full + s, (uint32_t)(np * (A_PIECE + B_PIECE)));
        for (int p = 0; p < np; ++p) tma_load_3d(&tmA, st + p * A_PIECE, full + s, kb * TK, m0, p);
        for (int p = 0; p < np; ++p)
          tma_load_3d(&tmB, st + MAXP * A_PIECE + p * B_PIECE, full + s, kb * TK, n0, p);
        issued = g + 1;
      }
      // Wait until the last slabs have been consumed (their slots released by the
      // MMAs' completion), so that no mbarrier arrival is still in flight when the
      // CTA exits; on the abort path, wait for the copies in flight to land instead.
      for (long long g = issued > STAGES ? issued - STAGES : 0; g < issued; ++g) {
        const int s = (int)(g % STAGES);
        const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
        unsigned long long t0 = gtimer();
        if (ok) {
          if (!mbar_wait(empty + s, ph, cta_abort, gerr)) ok = false;
        }
        if (!ok) {
          while (!mbar_try_wait(full + s, ph))
            if (gtimer() - t0 > WAIT_NS) break;
        }
      }
    }
    __syncwarp();
  } else if (warp == W_MMA) {
    if (lane == 0) {
      // ---------------- MMA issuer: chunk = CHUNK_SLABS consecutive K slabs of a tile;
      // first the small terms of every slab of the chunk, then its leading terms
      constexpr uint32_t idesc = idesc_bf16_f32(TM, TN);
      const int nch = (kslabs + CHUNK_SLABS - 1) / CHUNK_SLABS;
      bool ok = true;
      long long g = 0, gc = 0;   // slabs and chunks of this CTA so far
      for (long long i = 0; i < my_tiles && ok; ++i) {
        for (int ch = 0; ch < nch && ok; ++ch, ++gc) {
          const int b = (int)(gc & 1);
          if (gc >= 2 && !mbar_wait(tempty + b, (uint32_t)((gc >> 1) - 1) & 1u, cta_abort, gerr)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int ns = min(CHUNK_SLABS, kslabs - ch * CHUNK_SLABS);
          const uint32_t dst = tmem + (uint32_t)(b * TN);
          bool first = true;
          for (int pass = 0; pass < 2 && ok; ++pass) {
            const int t0 = pass == 0 ? 0 : terms.nsmall, t1 = pass == 0 ? terms.nsmall : terms.nterms;
            for (int q = 0; q < ns; ++q) {
              const long long gs = g + q;
              const int s = (int)(gs % STAGES);
              if (pass == 0) {   // a slab is waited for once, before its first MMA
                if (!mbar_wait(full + s, (uint32_t)(gs / STAGES) & 1u, cta_abort, gerr)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
              }
              const uint32_t st = su32(smem + s * STAGE_BYTES);
              for (int t = t0; t < t1; ++t) {
                const int pa_t = (int)(terms.code >> (4 * t)) & 3, pb_t = (int)(terms.code >> (4 * t + 2)) & 3;
                const uint64_t a0 = sdesc_sw(st + pa_t * A_PIECE);
                const uint64_t b0 = sdesc_sw(st + MAXP * A_PIECE + pb_t * B_PIECE);
#pragma unroll
                for (int kk = 0; kk < TK / 16; ++kk) {
                  // advance 16 BF16 = 32 bytes along K inside the swizzled row;
                  // the first MMA of a chunk starts the buffer from zero
                  umma_bf16(dst, a0 + (uint64_t)(2 * kk), b0 + (uint64_t)(2 * kk), idesc, first ? 0u : 1u);
                  first = false;
                }
              }
            }
          }
          if (!ok) break;
          for (int q = 0; q < ns; ++q) umma_commit(empty + (int)((g + q) % STAGES));   // slots free
          umma_commit(tfull + b);    // the chunk is complete
          g += ns;
        }
      }
      if (*cta_abort || *gerr) {
        // wait (bounded) until every MMA issued so far has completed, so that
        // TMEM is never released under a running MMA
        umma_commit(drain);
        unsigned long long t0 = gtimer();
        while (!mbar_try_wait(drain, 0))
          if (gtimer() - t0 > WAIT_NS) break;
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue warps: chunk partials -> FP32 registers -> C
    const int quarter = warp & 3, part = warp >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(part * EPI_COLS);
    bool ok = true;
    const int nch = (kslabs + CHUNK_SLABS - 1) / CHUNK_SLABS;
    long long g = 0;   // chunks of this CTA so far
    for (long long i = 0; i < my_tiles && ok; ++i) {
      const long long tile = blockIdx.x + i * gridDim.x;
      float acc[EPI_COLS];
#pragma unroll
      for (int j = 0; j < EPI_COLS; ++j) acc[j] = 0.0f;
      for (int kb = 0; kb < nch; ++kb, ++g) {
        const int b = (int)(g & 1);
        if (!mbar_wait(tfull + b, (uint32_t)(g >> 1) & 1u, cta_abort, gerr)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // two loads in flight per wait
#pragma unroll
        for (int q = 0; q < EPI_COLS; q += 2 * LD_COLS) {
          uint32_t v0[LD_COLS], v1[LD_COLS];
          tmem_ld_async(lane_base + (uint32_t)(b * TN + q), v0);
          tmem_ld_async(lane_base + (uint32_t)(b * TN + q + LD_COLS), v1);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < LD_COLS; ++j) acc[q + j] += __uint_as_float(v0[j]);
#pragma unroll
          for (int j = 0; j < LD_COLS; ++j) acc[q + LD_COLS + j] += __uint_as_float(v1[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(tempty + b)) : "memory");
      }
      if (!ok || *cta_abort) break;
      // the TMEM buffers are free again: the next tile's MMAs run while this one is stored
      const int row = (int)(tile % mtiles) * TM + quarter * 32 + lane;
      const int col0 = (int)(tile / mtiles) * TN + part * EPI_COLS;
      if (row < M) {
        float* dst = C + (long long)row * ldc + col0;
        const bool vec = ((ldc & 3) == 0) && ((((uintptr_t)C) & 15) == 0) && (col0 + EPI_COLS <= N);
        if (vec) {
#pragma unroll
          for (int j = 0; j < EPI_COLS; j += 4)
            *reinterpret_cast<float4*>(dst + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < EPI_COLS; ++j)
            if (col0 + j < N) dst[j] = acc[j];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == W_MMA) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// CTA-pair form (cta_group::2): a cluster of two CTAs on two SMs computes a 256 x 256
// tile of C with M = 256 MMAs issued by CTA 0.  CTA r holds rows 128 r .. of the A
// tile and rows 128 r .. of the B tile (N) in its own shared memory, so each SM
// receives half of B; K slabs of 128-byte rows (128-byte swizzle), every piece of a
// slab in one ring stage.  The ring holds six 32 KiB units (one piece of A and one of
// B): 6 / npieces stages, so forms with fewer pieces keep more slabs in flight.
// CTA r's TMEM holds rows
// 128 r .. of the accumulator.  CTA 1's copies complete on its own barrier; a thread
// of CTA 1 then arrives on CTA 0's barrier, whose MMA thread waits for both.  The
// MMA completions arrive on the ring and accumulator barriers of both CTAs.
// ---------------------------------------------------------------------------
#ifndef HOTRG_TC_USE_PAIR
#define HOTRG_TC_USE_PAIR 1
#endif
namespace {
constexpr int P_TK = 64, P_UNITS = 6, P_MAXST = 6;
constexpr int P_A_PIECE = 128 * P_TK * 2;                    // 16 KiB: this CTA's A rows
constexpr int P_B_PIECE = 128 * P_TK * 2;                    // 16 KiB: this CTA's B rows
constexpr int P_UNIT = P_A_PIECE + P_B_PIECE;                // one piece of each operand
constexpr int P_SMEM = 1024 + P_UNITS * P_UNIT + 256;
constexpr int P_NTHREADS = 320;                              // 8 epilogue warps + producer + MMA/relay
static_assert(P_SMEM <= 227 * 1024, "shared memory of one CTA");
}  // namespace

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// arrival on the mbarrier at bar's offset in CTA `rank` of the cluster
__device__ __forceinline__ void mbar_arrive_rank(uint64_t* bar, uint32_t rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(su32(bar)), "r"(rank));
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}

__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

template <bool TF32>
__device__ __forceinline__ void umma_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  if (TF32)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrives on the mbarrier at bar's offset in every CTA of cta_mask once the pair MMAs
// issued so far by this thread have completed
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar, uint16_t cta_mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          su32(bar)),
      "h"(cta_mask)
      : "memory");
}

template <bool TF32>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(P_NTHREADS, 1)
    tc_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        float* __restrict__ C, int M, int N, long long ldc, int kslabs, TcTerms terms,
                        int* g_err) {
  extern __shared__ uint8_t smem_raw[];
  volatile int* gerr = g_err;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + P_UNITS * P_UNIT);
  uint64_t* empty = full + P_MAXST;
  uint64_t* tfull = empty + P_MAXST;     // [2] MMA -> epilogue (both CTAs)
  uint64_t* tempty = tfull + 2;          // [2] epilogue of both CTAs -> MMA (CTA 0)
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* cta_abort = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const bool leader = rank == 0;
  const int mgroups = (M + 255) / 256;
  const long long ngroups = (long long)mgroups * ((N + 255) / 256);
  const long long cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const long long tiles_here = ngroups > cid ? (ngroups - 1 - cid) / ncl + 1 : 0;
  auto grp = [&](long long i) { return cid + i * ncl; };
  const int np = terms.npieces;
  const int nst = P_UNITS / np;                 // ring stages
  const int stage_bytes = np * P_UNIT;          // A pieces, then B pieces

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(full + s, leader ? 2 : 1);   // CTA 0: its own copies and CTA 1's relay
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, 16);             // the 8 epilogue warps of each CTA
    }
    mbar_init(drain, 1);
    *cta_abort = *gerr ? 1 : 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmB) : "memory");
  }
  if (warp == 9) {
    // one warp of each CTA of the pair allocates, collectively, the TMEM of both
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();   // both CTAs' barriers and TMEM exist before any copy or arrival
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const long long my_tiles = *cta_abort ? 0 : tiles_here;
  const long long total = my_tiles * kslabs;

  if (warp == 8) {
    if (lane == 0) {
      // ---------------- TMA producer (both CTAs): this CTA's A rows and B rows
      long long issued = 0;
      bool ok = true;
      for (long long g = 0; g < total; ++g) {
        const int s = (int)(g % nst);
        const uint32_t ph = (uint32_t)(g / nst) & 1u;
        if (!mbar_wait(empty + s, ph ^ 1u, cta_abort, gerr)) {
          ok = false;
          break;
        }
        const long long gg = grp(g / kslabs);
        const int kb = (int)(g % kslabs);
        const int m0 = (int)(gg % mgroups) * 256 + (int)rank * 128;
        const int nb0 = (int)(gg / mgroups) * 256 + (int)rank * 128;
        const int k0 = kb * (TF32 ? P_TK / 2 : P_TK);   // elements of a 128-byte row
        uint8_t* st = smem + s * stage_bytes;
        mbar_expect_tx(full + s, (uint32_t)stage_bytes);
        for (int p = 0; p < np; ++p) tma_load_3d(&tmA, st + p * P_A_PIECE, full + s, k0, m0, p);
        for (int p = 0; p < np; ++p)
          tma_load_3d(&tmB, st + np * P_A_PIECE + p * P_B_PIECE, full + s, k0, nb0, p);
        issued = g + 1;
      }
      for (long long g = issued > nst ? issued - nst : 0; g < issued; ++g) {
        const int s = (int)(g % nst);
        const uint32_t ph = (uint32_t)(g / nst) & 1u;
        unsigned long long t0 = gtimer();
        if (ok && !mbar_wait(empty + s, ph, cta_abort, gerr)) ok = false;
        if (!ok)
          while (!mbar_try_wait(full + s, ph))
            if (gtimer() - t0 > WAIT_NS) break;
      }
    }
    __syncwarp();
  } else if (warp == 9) {
    if (lane == 0 && !leader) {
      // ---------------- relay (CTA 1): each slab of this CTA has landed -> CTA 0
      for (long long g = 0; g < total; ++g) {
        const int s = (int)(g % nst);
        if (!mbar_wait(full + s, (uint32_t)(g / nst) & 1u, cta_abort, gerr)) break;
        mbar_arrive_rank(full + s, 0);
      }
    } else if (lane == 0) {
      // ---------------- MMA issuer (CTA 0): M = 256, N = 256, K = 32 bytes of a row;
      // one chunk per slab, its small terms first
      constexpr uint32_t idesc = TF32 ? idesc_tf32_f32(256, 256) : idesc_bf16_f32(256, 256);
      bool ok = true;
      for (long long g = 0; g < total && ok; ++g) {
        const int b = (int)(g & 1);
        if (g >= 2 && !mbar_wait(tempty + b, (uint32_t)((g >> 1) - 1) & 1u, cta_abort, gerr)) break;
        tc_fence_after();
        const int s = (int)(g % nst);
        if (!mbar_wait(full + s, (uint32_t)(g / nst) & 1u, cta_abort, gerr)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dst = tmem + (uint32_t)(b * 256);
        const uint32_t st = su32(smem + s * stage_bytes);
        for (int t = 0; t < terms.nterms; ++t) {
          const int pa_t = (int)(terms.code >> (4 * t)) & 3, pb_t = (int)(terms.code >> (4 * t + 2)) & 3;
          const uint64_t a0 = sdesc_sw128(st + pa_t * P_A_PIECE);
          const uint64_t b0 = sdesc_sw128(st + np * P_A_PIECE + pb_t * P_B_PIECE);
#pragma unroll
          for (int kk = 0; kk < P_TK / 16; ++kk)   // 32 bytes (2 descriptor units) per MMA
            umma_pair<TF32>(dst, a0 + (uint64_t)(2 * kk), b0 + (uint64_t)(2 * kk), idesc,
                            (t != 0 || kk != 0) ? 1u : 0u);
        }
        umma_commit_pair(empty + s, (uint16_t)0x3);   // the slot of both CTAs is free
        umma_commit_pair(tfull + b, (uint16_t)0x3);   // the chunk is in both CTAs' TMEM
      }
      if (*cta_abort || *gerr) {
        asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(drain))
                     : "memory");
        unsigned long long t0 = gtimer();
        while (!mbar_try_wait(drain, 0))
          if (gtimer() - t0 > WAIT_NS) break;
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue warps (both CTAs): this CTA's 128 rows of the tile
    const int quarter = warp & 3, part = warp >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(part * 128);
    bool ok = true;
    long long g = 0;
    for (long long i = 0; i < my_tiles && ok; ++i) {
      float acc[128];
#pragma unroll
      for (int j = 0; j < 128; ++j) acc[j] = 0.0f;
      for (int kb = 0; kb < kslabs; ++kb, ++g) {
        const int b = (int)(g & 1);
        if (!mbar_wait(tfull + b, (uint32_t)(g >> 1) & 1u, cta_abort, gerr)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int q = 0; q < 128; q += 64) {
          uint32_t v0[32], v1[32];
          tmem_ld_async(lane_base + (uint32_t)(b * 256 + q), v0);
          tmem_ld_async(lane_base + (uint32_t)(b * 256 + q + 32), v1);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 32; ++j) acc[q + j] += __uint_as_float(v0[j]);
#pragma unroll
          for (int j = 0; j < 32; ++j) acc[q + 32 + j] += __uint_as_float(v1[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_rank(tempty + b, 0);
      }
      if (!ok || *cta_abort) break;
      const long long gg = grp(i);
      const int row = (int)(gg % mgroups) * 256 + (int)rank * 128 + quarter * 32 + lane;
      const int col0 = (int)(gg / mgroups) * 256 + part * 128;
      if (row < M) {
        float* dst = C + (long long)row * ldc + col0;
        const bool vec = ((ldc & 3) == 0) && ((((uintptr_t)C) & 15) == 0) && (col0 + 128 <= N);
        if (vec) {
#pragma unroll
          for (int j = 0; j < 128; j += 4)
            *reinterpret_cast<float4*>(dst + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 128; ++j)
            if (col0 + j < N) dst[j] = acc[j];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();   // no CTA leaves while its peer may still use its TMEM or barriers
  if (warp == 9) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return nullptr;
  }();
  return fn;
}

int tc_gemm_ready() { return get_encode() != nullptr; }

// operand pieces stored as [piece][rows][kpad] elements (BF16, or TF32 in FP32 words);
// one box = box_k elements of K (box_k x element size = the swizzle width) x box_rows
// rows of one piece
static int make_map(CUtensorMap* map, const void* base, int rows, int kpad, int npieces, int box_rows,
                    int box_k = TK, bool tf32 = false) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return -1;
  const cuuint64_t esz = tf32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)npieces};
  cuuint64_t strides[2] = {(cuuint64_t)kpad * esz, (cuuint64_t)kpad * esz * (cuuint64_t)rows};
  cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base,
                   dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   box_k * esz == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    fprintf(stderr, "hotrg: tensor map encoding failed (CUresult %d; rows %d, kpad %d)\n", (int)r, rows,
            kpad);
    return -1;
  }
  return 0;
}

// The kernel's dynamic shared-memory limit, raised once per device.
static bool gemm_smem_attr_set() {
  static std::atomic<int> done[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (dev >= 0 && dev < kMaxDevices && done[dev].load(std::memory_order_acquire)) return true;
  if (cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) !=
      cudaSuccess)
    return false;
  if (dev >= 0 && dev < kMaxDevices) done[dev].store(1, std::memory_order_release);
  return true;
}

static bool pair_smem_attr_set() {
  static std::atomic<int> done[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (dev >= 0 && dev < kMaxDevices && done[dev].load(std::memory_order_acquire)) return true;
  if (cudaFuncSetAttribute(tc_gemm_pair_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM) !=
          cudaSuccess ||
      cudaFuncSetAttribute(tc_gemm_pair_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM) !=
          cudaSuccess)
    return false;
  if (dev >= 0 && dev < kMaxDevices) done[dev].store(1, std::memory_order_release);
  return true;
}

int launch_tc_gemm(const void* A, int M, const void* B, int N, int Kpad, int npieces, int nterms,
                   const int* pa, const int* pb, float* C, long long ldc, int* err_flag, cudaStream_t s,
                   float* ms_out, int pfmt) {
  const bool tf32 = pfmt == PIECE_TF32;
  // TF32 pieces: 32-element (128-byte) slabs in the pair form only
  if (Kpad % (tf32 ? P_TK / 2 : TK) != 0 || Kpad < TK || nterms < 1 || nterms > 9 || npieces < 1 ||
      npieces > MAXP || M < 1 || N < 1 || (pfmt != PIECE_BF16 && !tf32) || (tf32 && !HOTRG_TC_USE_PAIR) ||
      (((uintptr_t)A) & 15) || (((uintptr_t)B) & 15)) {
    fprintf(stderr, "hotrg: GEMM arguments rejected (M %d, N %d, Kpad %d, pieces %d, terms %d, format %d, A %p, B %p)\n",
            M, N, Kpad, npieces, nterms, pfmt, A, B);
    return -1;
  }
  {
    const cudaError_t pre = cudaGetLastError();
    if (pre != cudaSuccess) {
      fprintf(stderr, "hotrg: CUDA error pending before the GEMM launch: %s\n", cudaGetErrorString(pre));
      return -1;
    }
  }
  const bool use_pair = tf32 || (HOTRG_TC_USE_PAIR != 0 && Kpad % P_TK == 0);
  const int slab_k = tf32 ? P_TK / 2 : P_TK;   // elements of a 128-byte row
  CUtensorMap ma, mb;
  if (use_pair) {
    if (make_map(&ma, A, M, Kpad, npieces, 128, slab_k, tf32) || make_map(&mb, B, N, Kpad, npieces, 128, slab_k, tf32))
      return -1;
  } else if (make_map(&ma, A, M, Kpad, npieces, TM) || make_map(&mb, B, N, Kpad, npieces, TN)) {
    return -1;
  }
  // terms ordered by decreasing piece order (pa + pb): the smallest terms go first into
  // the zeroed accumulator of a chunk, the leading term x_0 y_0 last
  TcTerms terms;
  terms.nterms = nterms;
  terms.npieces = npieces;
  terms.nsmall = 0;
  int order[9];
  for (int t = 0; t < nterms; ++t) order[t] = t;
  std::stable_sort(order, order + nterms,
                   [&](int x, int y) { return pa[x] + pb[x] > pa[y] + pb[y]; });
  terms.code = 0;
  for (int t = 0; t < nterms; ++t) {
    const int a = pa[order[t]], b = pb[order[t]];
    if (a < 0 || a >= npieces || b < 0 || b >= npieces) {
      fprintf(stderr, "hotrg: GEMM term %d uses a piece beyond %d\n", t, npieces);
      return -1;
    }
    terms.code |= (unsigned long long)(a | (b << 2)) << (4 * t);
    if (a + b > 0) terms.nsmall = t + 1;
  }
  if (use_pair ? !pair_smem_attr_set() : !gemm_smem_attr_set()) {
    fprintf(stderr, "hotrg: GEMM shared-memory attribute refused\n");
    return -1;
  }
  const long long ntiles = (long long)((M + TM - 1) / TM) * ((N + TN - 1) / TN);
  const long long ngroups = (long long)((M + 255) / 256) * ((N + 255) / 256);
  const int grid = use_pair ? 2 * (int)std::min<long long>(ngroups, std::max(1, sm_count() / 2))
                            : (int)std::min<long long>(ntiles, sm_count());
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms_out) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  if (use_pair && tf32)
    tc_gemm_pair_kernel<true><<<grid, P_NTHREADS, P_SMEM, s>>>(ma, mb, C, M, N, ldc, Kpad / slab_k, terms, err_flag);
  else if (use_pair)
    tc_gemm_pair_kernel<false><<<grid, P_NTHREADS, P_SMEM, s>>>(ma, mb, C, M, N, ldc, Kpad / slab_k, terms, err_flag);
  else
    tc_gemm_kernel<<<grid, NTHREADS, SMEM_BYTES, s>>>(ma, mb, C, M, N, ldc, Kpad / TK, terms, err_flag);
  ++g_launches;
  if (ms_out) {
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms_out, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "hotrg: GEMM launch error %s (grid %d)\n", cudaGetErrorString(e), grid);
    return -1;
  }
  return 0;
}

// Operand pieces for the rate probe: small multiples of 1/8 (exact in BF16 and in
// TF32) from a hash
__global__ void fill_pieces_kernel(void* p, long long n, unsigned seed, int tf32) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned x = (unsigned)i * 2654435761u ^ seed;
    x ^= x >> 15;
    x *= 2246822519u;
    x ^= x >> 13;
    const float v = (float)((int)(x % 17u) - 8) * 0.125f;
    if (tf32)
      ((float*)p)[i] = v;
    else
      ((__nv_bfloat16*)p)[i] = __float2bfloat16(v);
  }
}

int measure_tc_gemm_rate(int npieces, int M, int N, int Kpad, int iters, double* ms_per_launch, int pfmt) {
  const bool tf32 = pfmt == PIECE_TF32;
  if (npieces < (tf32 ? 1 : 2) || npieces > (tf32 ? 2 : MAXP) || M < 1 || N < 1 || Kpad < TK || Kpad % TK ||
      iters < 1)
    return -1;
  void *A = nullptr, *B = nullptr;
  float* C = nullptr;
  int* err = nullptr;
  const long long esz = tf32 ? 4 : 2;
  const long long na = (long long)npieces * M * Kpad, nb = (long long)npieces * N * Kpad;
  if (cudaMalloc(&A, esz * na) != cudaSuccess || cudaMalloc(&B, esz * nb) != cudaSuccess ||
      cudaMalloc(&C, 4LL * M * N) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(A);
    cudaFree(B);
    cudaFree(C);
    cudaFree(err);
    return -2;
  }
  cudaMemset(err, 0, sizeof(int));
  fill_pieces_kernel<<<4 * sm_count(), 256>>>(A, na, 1u, tf32 ? 1 : 0);
  fill_pieces_kernel<<<4 * sm_count(), 256>>>(B, nb, 2u, tf32 ? 1 : 0);
  g_launches += 2;
  int ta[6], tb[6];
  const int nt = split_terms(npieces, ta, tb);
  int r = launch_tc_gemm(A, M, B, N, Kpad, npieces, nt, ta, tb, C, N, err, 0, nullptr, pfmt);   // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, 0);
  for (int i = 0; i < iters && r == 0; ++i)
    r = launch_tc_gemm(A, M, B, N, Kpad, npieces, nt, ta, tb, C, N, err, 0, nullptr, pfmt);
  cudaEventRecord(e1, 0);
  cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  int h_err = 0;
  cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(A);
  cudaFree(B);
  cudaFree(C);
  cudaFree(err);
  if (r != 0 || cudaGetLastError() != cudaSuccess) return -3;
  if (h_err) return h_err;
  *ms_per_launch = ms / iters;
  return 0;
}

}  // namespace hotrg
