// Bottleneck contraction (Sec. 4.2.9, Eq. BottleneckPart) on the 5th-generation
// tensor cores:
//   C[(c, n^), (n', n~)] = sum_{(rho, n^')} T[(c, n^), (rho, n^')] B[(n', n~), (rho, n^')]
// with both operands split into BF16 pieces, x = x_0 + x_1 (+ x_2), and the
// product formed as a sum of piece products (terms).
//
// One CTA computes a 128 x 256 tile of C.  Warp 8 (one lane) streams 64-wide
// K slabs of the A and B pieces into a 4-stage shared-memory ring with TMA
// (128-byte swizzle).  Warp 9 (one lane) issues tcgen05.mma (M=128, N=256,
// K=16, kind::f16, BF16 x BF16 -> FP32) and releases ring slots with
// tcgen05.commit.  The tensor core's FP32 accumulation truncates, so a long
// accumulation drifts towards zero; the K loop is therefore cut into short
// chunks, each accumulated from zero into one of two TMEM buffers (256
// columns each, used alternately), while warps 0-7 drain the other buffer
// with tcgen05.ld (warp w owns TMEM lanes 32(w%4).. and columns 128(w/4)..)
// and add the chunk into FP32 registers with round-to-nearest.  Every
// mbarrier wait is bounded in time; an expired wait sets a global error flag
// that also makes the CTAs still to come exit at once.
#include <cuda.h>
#include <stdio.h>
#include <stdlib.h>

#include "hotrg_internal.cuh"
#include "../../include/hotrg.h"

namespace hotrg {

namespace {
constexpr int TM = 128, TN = 256, TK = 64, STAGES = 4;
constexpr int A_STAGE = TM * TK * 2;   // 16 KiB
constexpr int B_STAGE = TN * TK * 2;   // 32 KiB
constexpr int TMEM_COLS = 512;         // two 256-column FP32 accumulators
constexpr int NTHREADS = 320;          // 8 epilogue warps + producer + MMA
constexpr int SMEM_BYTES = 1024 + STAGES * (A_STAGE + B_STAGE) + 256;
constexpr unsigned long long WAIT_NS = 4000000000ull;  // 4 s per wait
}  // namespace

struct TcTerms {
  int nterms;
  int pa[9];
  int pb[9];
  int clen[9];   // K-blocks per accumulation chunk of each term
};

// chunks of term t: ceil(kblocks / clen[t])
__device__ __forceinline__ int count_chunks(const TcTerms& terms, int kblocks) {
  int n = 0;
  for (int t = 0; t < terms.nterms; ++t) n += (kblocks + terms.clen[t] - 1) / terms.clen[t];
  return n;
}

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

// Shared-memory matrix descriptor for a K-major operand tile written by TMA
// with the 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, N, M.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
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

// 32 lanes x 32 columns of FP32 from TMEM; the values are usable after tmem_wait_ld()
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&v)[32]) {
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

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   float* __restrict__ C, int M, int N, long long ldc, int kblocks, TcTerms terms,
                   int* g_err) {
  extern __shared__ uint8_t smem_raw[];
  volatile int* gerr = g_err;
  if (*gerr) return;  // an earlier CTA gave up: do nothing
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_STAGE;
  uint64_t* full = (uint64_t*)(sB + STAGES * B_STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;      // [2] MMA -> epilogue
  uint64_t* tempty = tfull + 2;          // [2] epilogue -> MMA
  uint64_t* drain = tempty + 2;          // MMA completion on the abort path
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* cta_abort = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  const int total = terms.nterms * kblocks;
  const int nchunks = count_chunks(terms, kblocks);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, 8);
    }
    mbar_init(drain, 1);
    *cta_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmB) : "memory");
  }
  if (warp == 9) {
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

  if (warp == 8) {
    if (lane == 0) {
      // ---------------- TMA producer
      int issued = 0;
      bool ok = true;
      for (int it = 0; it < total; ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        if (!mbar_wait(empty + s, ph ^ 1u, cta_abort, gerr)) {
          ok = false;
          break;
        }
        mbar_expect_tx(full + s, A_STAGE + B_STAGE);
        const int t = it / kblocks, kb = it - t * kblocks;
        tma_load_3d(&tmA, sA + s * A_STAGE, full + s, kb * TK, m0, terms.pa[t]);
        tma_load_3d(&tmB, sB + s * B_STAGE, full + s, kb * TK, n0, terms.pb[t]);
        issued = it + 1;
      }
      if (!ok) {
        // let the copies already in flight land before the CTA can exit
        for (int it = issued > STAGES ? issued - STAGES : 0; it < issued; ++it) {
          unsigned long long t0 = gtimer();
          while (!mbar_try_wait(full + (it % STAGES), (uint32_t)(it / STAGES) & 1u))
            if (gtimer() - t0 > WAIT_NS) break;
        }
      }
    }
    __syncwarp();
  } else if (warp == 9) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t idesc = idesc_bf16_f32(TM, TN);
      bool ok = true;
      int c = 0, t = 0, kb0 = 0;   // chunk c = K-blocks [kb0, kb0 + clen[t]) of term t
      for (; c < nchunks && ok; ++c) {
        const int b = c & 1;
        if (c >= 2 && !mbar_wait(tempty + b, (uint32_t)((c >> 1) - 1) & 1u, cta_abort, gerr)) break;
        tc_fence_after();
        const uint32_t dst = tmem + (uint32_t)(b * TN);
        const int it_begin = t * kblocks + kb0;
        const int it_end = t * kblocks + min(kblocks, kb0 + terms.clen[t]);
        kb0 += terms.clen[t];
        if (kb0 >= kblocks) {
          kb0 = 0;
          ++t;
        }
        for (int it = it_begin; it < it_end; ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (!mbar_wait(full + s, ph, cta_abort, gerr)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t a0 = sdesc_sw128(su32(sA + s * A_STAGE));
          const uint64_t b0 = sdesc_sw128(su32(sB + s * B_STAGE));
#pragma unroll
          for (int kk = 0; kk < TK / 16; ++kk) {
            // advance 16 BF16 = 32 bytes along K inside the 128-byte swizzled row;
            // the first MMA of a chunk starts the buffer from zero
            umma_bf16(dst, a0 + (uint64_t)(2 * kk), b0 + (uint64_t)(2 * kk), idesc,
                      (it != it_begin || kk != 0) ? 1u : 0u);
          }
          umma_commit(empty + s);
        }
        // arrives once every MMA of this chunk has completed
        if (ok) umma_commit(tfull + b);
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
    // ---------------- epilogue warps 0-7: chunk partials -> FP32 registers
    const int quarter = warp & 3, half = warp >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 128);
    float acc[128];
#pragma unroll
    for (int j = 0; j < 128; ++j) acc[j] = 0.0f;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int b = c & 1;
      if (!mbar_wait(tfull + b, (uint32_t)(c >> 1) & 1u, cta_abort, gerr)) {
        ok = false;
        break;
      }
      tc_fence_after();
      // two 32-column loads in flight per wait
#pragma unroll
      for (int q = 0; q < 4; q += 2) {
        uint32_t v0[32], v1[32];
        tmem_ld32_async(lane_base + (uint32_t)(b * TN + q * 32), v0);
        tmem_ld32_async(lane_base + (uint32_t)(b * TN + (q + 1) * 32), v1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[q * 32 + j] += __uint_as_float(v0[j]);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[(q + 1) * 32 + j] += __uint_as_float(v1[j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(tempty + b)) : "memory");
    }
    if (ok && !*cta_abort) {
      const int row = m0 + quarter * 32 + lane;
      const int col0 = n0 + half * 128;
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
  if (warp == 9) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
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

// K-blocks (of 64) of the leading term x_0 y_0 accumulated in TMEM before the
// epilogue adds them into FP32 registers.  Tuning knob HOTRG_TC_CHUNK_KBLOCKS
// (default 2 = K chunks of 128: the truncating tensor-core accumulation then
// spans 8 MMAs only).  The terms of order 2^-8 (x_1 y_0, x_0 y_1) take chunks 8
// times longer and those of order 2^-16 the whole K at once: measured on 4D Ising
// chi=6, this leaves ln Z/V where uniform chunks put it (8.4e-8 against 8.3e-8),
// while the leading chunk's length does move it.
int tc_chunk_kblocks() {
  static const int v = [] {
    const char* e = getenv("HOTRG_TC_CHUNK_KBLOCKS");
    const int x = e ? atoi(e) : 2;
    return x < 1 ? 1 : x;
  }();
  return v;
}

// operand pieces stored as [piece][rows][kpad] BF16
static int make_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int kpad, int npieces,
                    int box_rows) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return -1;
  cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)npieces};
  cuuint64_t strides[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)kpad * 2 * (cuuint64_t)rows};
  cuuint32_t box[3] = {(cuuint32_t)TK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    fprintf(stderr, "hotrg: tensor map encoding failed (CUresult %d; rows %d, kpad %d)\n", (int)r, rows,
            kpad);
    return -1;
  }
  return 0;
}

int launch_tc_gemm(const __nv_bfloat16* A, int M, const __nv_bfloat16* B, int N, int Kpad,
                   int npieces, int nterms, const int* pa, const int* pb, float* C, long long ldc,
                   int* err_flag, cudaStream_t s, float* ms_out, int chunk_kblocks) {
  if (Kpad % TK != 0 || nterms < 1 || nterms > 9 || (((uintptr_t)A) & 15) || (((uintptr_t)B) & 15)) {
    fprintf(stderr, "hotrg: GEMM arguments rejected (Kpad %d, terms %d, A %p, B %p)\n", Kpad, nterms,
            (const void*)A, (const void*)B);
    return -1;
  }
  {
    const cudaError_t pre = cudaGetLastError();
    if (pre != cudaSuccess) {
      fprintf(stderr, "hotrg: CUDA error pending before the GEMM launch: %s\n", cudaGetErrorString(pre));
      return -1;
    }
  }
  CUtensorMap ma, mb;
  if (make_map(&ma, A, M, Kpad, npieces, TM) || make_map(&mb, B, N, Kpad, npieces, TN)) return -1;
  TcTerms terms;
  terms.nterms = nterms;
  const int kblocks = Kpad / TK, base = chunk_kblocks > 0 ? chunk_kblocks : tc_chunk_kblocks();
  for (int t = 0; t < 9; ++t) {
    terms.pa[t] = t < nterms ? pa[t] : 0;
    terms.pb[t] = t < nterms ? pb[t] : 0;
    const int order = terms.pa[t] + terms.pb[t];
    terms.clen[t] = order == 0 ? base : order == 1 ? 8 * base : kblocks;
    if (terms.clen[t] < 1) terms.clen[t] = 1;
  }
  static const bool attr = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                SMEM_BYTES) == cudaSuccess;
  (void)attr;
  dim3 grid((M + TM - 1) / TM, (N + TN - 1) / TN);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms_out) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  tc_gemm_kernel<<<grid, NTHREADS, SMEM_BYTES, s>>>(ma, mb, C, M, N, ldc, kblocks, terms, err_flag);
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
    fprintf(stderr, "hotrg: GEMM launch error %s (grid %u x %u)\n", cudaGetErrorString(e), grid.x, grid.y);
    return -1;
  }
  return 0;
}

}  // namespace hotrg
