// hotrg_gemm_nt_noalloc: the bottleneck GEMM for callers that must not
// allocate device memory.  Its scratch -- the BF16 pieces of both operands,
// the FP32 product and an error word -- lives in one file-scope __device__
// array of fixed size, so the call itself never allocates or frees.
#include <cuda_runtime.h>

#include <mutex>

#include "hotrg_internal.cuh"
#include "../../include/hotrg.h"

namespace hotrg {
namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // HOTRG_NOALLOC_SCRATCH_BYTES

// Every GPU that loads the library holds this array until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device; looked up once
// per device (host code cannot use the symbol itself as a device pointer).
unsigned char* scratch_on_current_device(int* status) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    *status = HOTRG_ECUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      *status = HOTRG_ECUDA;
      return nullptr;
    }
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  *status = HOTRG_OK;
  return g_scratch_ptr[dev];
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

__global__ void widen_kernel(const float* __restrict__ in, double* __restrict__ out, long long n) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = (double)in[i];
}

}  // namespace
}  // namespace hotrg

using namespace hotrg;

extern "C" int hotrg_gemm_nt_noalloc(int mode, int M, int N, int K, const double* A, const double* B,
                                     double* C, void* stream) {
  // the size limits of hotrg_gemm_nt, so that bad sizes give HOTRG_EINVAL in every mode
  if (mode < HOTRG_PREC_FP64 || mode > HOTRG_PREC_BF16X6 || M < 1 || N < 1 || K < 1 || M > (1 << 20) ||
      N > (1 << 20) || K > (1 << 20) || !A || !B || !C)
    return HOTRG_EINVAL;
  if ((long long)M * K > (1LL << 31) || (long long)N * K > (1LL << 31) || (long long)M * N > (1LL << 31))
    return HOTRG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int status = HOTRG_OK;
  unsigned char* base = scratch_on_current_device(&status);
  if (!base) return status;

  const int np = mode == HOTRG_PREC_BF16X3 ? 2 : 3;
  const long long Kpad = ((long long)K + 63) / 64 * 64;
  // scratch layout: [error word][A pieces][B pieces][FP32 product]
  const size_t off_a = 256;
  const size_t bytes_a = align256(sizeof(__nv_bfloat16) * np * (size_t)M * Kpad);
  const size_t off_b = off_a + bytes_a;
  const size_t bytes_b = align256(sizeof(__nv_bfloat16) * np * (size_t)N * Kpad);
  const size_t off_c = off_b + bytes_b;
  const size_t bytes_c = align256(sizeof(float) * (size_t)M * N);
  if (mode != HOTRG_PREC_FP64 && off_c + bytes_c > kScratchBytes) return HOTRG_EINVAL;

  int* err = (int*)base;
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) status = HOTRG_ECUDA;
  if (status == HOTRG_OK && mode == HOTRG_PREC_FP64) {
    launch_gemm_nt_f64(A, K, B, K, C, N, 0, M, N, K, 1, 0, s);
  } else if (status == HOTRG_OK) {
    __nv_bfloat16* pa = (__nv_bfloat16*)(base + off_a);
    __nv_bfloat16* pb = (__nv_bfloat16*)(base + off_b);
    float* c32 = (float*)(base + off_c);
    // the pieces keep the previous call's contents: the K padding must read as zero
    if (Kpad != K) {
      if (cudaMemsetAsync(pa, 0, bytes_a, s) != cudaSuccess || cudaMemsetAsync(pb, 0, bytes_b, s) != cudaSuccess)
        status = HOTRG_ECUDA;
    }
    if (status == HOTRG_OK) {
      launch_split(A, M, K, K, pa, Kpad, (long long)M * Kpad, np, PIECE_BF16, s);
      launch_split(B, N, K, K, pb, Kpad, (long long)N * Kpad, np, PIECE_BF16, s);
      int ta[6], tb[6];
      const int nt = split_terms(np, ta, tb);
      if (launch_tc_gemm(pa, M, pb, N, (int)Kpad, np, nt, ta, tb, c32, N, err, s, nullptr, PIECE_BF16) != 0)
        status = HOTRG_ECUDA;
    }
    if (status == HOTRG_OK) {
      long long n = (long long)M * N;
      long long blocks = (n + 255) / 256;
      const long long cap = 16LL * sm_count();
      if (blocks > cap) blocks = cap;
      widen_kernel<<<(unsigned)blocks, 256, 0, s>>>(c32, C, n);
      ++g_launches;
    }
  }
  int e = 0;
  if (status == HOTRG_OK && cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    status = HOTRG_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) status = HOTRG_ECUDA;
  if (cudaGetLastError() != cudaSuccess && status == HOTRG_OK) status = HOTRG_ECUDA;
  if (status == HOTRG_OK && e != 0) status = e;
  return status;
}
