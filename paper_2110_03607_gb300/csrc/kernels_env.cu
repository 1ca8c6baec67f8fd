// FP64 environment build (Sec. 3.2, Eqs. Aux_Tensor_hat_S / Aux_Tensor_check_S;
// Sec. 4.2.4) and the plain FP64 contraction GEMM.
//
// Each S tensor is a Gram matrix: with X = T permuted to [(n_j, rho) | rest],
// S_{(f rho),(g eta)} = sum_rest X[(f, rho), rest] X[(g, eta), rest].  The
// GEMM below computes C = A . B^T for K-contiguous A and B (an "NT" GEMM) in
// FP64 DFMA tiles, with split-K partial outputs so that every SM has work.
#include "hotrg_internal.cuh"

namespace hotrg {

namespace {
constexpr int BM = 64, BN = 64, BK = 16;
}

// C[z][i][j] = sum_{k in split z} A[i*lda + k] * B[j*ldb + k], in T x T tiles (T = 64 for
// the large products, 32 for the symmetric Gram blocks, whose diagonal tiles are half
// wasted and whose sizes sit just above multiples of 64 at zero field); 256 threads,
// (T/16) x (T/16) outputs each.
template <int T>
__global__ void __launch_bounds__(256, 2) gemm_nt_f64_kernel(
    const double* __restrict__ A, long long lda, const double* __restrict__ B, long long ldb,
    double* __restrict__ C, long long ldc, long long split_stride, int M, int N, long long K,
    long long kchunk, int upper_only) {
  constexpr int R = T / 16;      // outputs per thread along each dim
  constexpr int L = T / 16;      // consecutive k loaded per thread per operand
  __shared__ double As[BK][T + 1];
  __shared__ double Bs[BK][T + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  int bx = blockIdx.x, by = blockIdx.y;
  if (upper_only) {
    // blockIdx.x enumerates the tile pairs (ti <= tj) of the upper triangle, row by row
    const int nt = (M + T - 1) / T;
    int t = blockIdx.x, ti = 0;
    while (t >= nt - ti) {
      t -= nt - ti;
      ++ti;
    }
    by = ti;
    bx = ti + t;
  }
  const int n0 = bx * T, m0 = by * T;
  // a diagonal tile of a symmetric product: output (ty + 16 i, tx + 16 j) with i > j lies
  // below the diagonal (tx - ty <= 15), which the reductions never read; skipped block-wide
  const bool diag = upper_only && bx == by;
  const long long k_lo = (long long)blockIdx.z * kchunk;
  long long k_hi = k_lo + kchunk;
  if (k_hi > K) k_hi = K;
  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.0;
  // loader mapping: T rows x 16 k; thread -> (row = tid / (16 / L), k = (tid % (16 / L)) * L .. +L-1).
  // The next slab is fetched into registers while the current one is multiplied.
  constexpr int TPR = 16 / L;    // threads per row
  const int lr = tid / TPR, lk = (tid % TPR) * L;
  const int ra = m0 + lr, rb = n0 + lr;
  double pa[L], pb[L];
  auto fetch = [&](long long k0) {
#pragma unroll
    for (int u = 0; u < L; ++u) {
      long long k = k0 + lk + u;
      pa[u] = (ra < M && k < k_hi) ? A[(long long)ra * lda + k] : 0.0;
      pb[u] = (rb < N && k < k_hi) ? B[(long long)rb * ldb + k] : 0.0;
    }
  };
  if (k_lo < k_hi) fetch(k_lo);
  for (long long k0 = k_lo; k0 < k_hi; k0 += BK) {
#pragma unroll
    for (int u = 0; u < L; ++u) {
      As[lk + u][lr] = pa[u];
      Bs[lk + u][lr] = pb[u];
    }
    __syncthreads();
    if (k0 + BK < k_hi) fetch(k0 + BK);
    // two bodies, so that the diagonal tiles' skipped products are not issued at all
    // (a predicated-off FMA would still take its slot in the FP64 pipe)
    if (diag) {
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double a[R], b[R];
#pragma unroll
        for (int i = 0; i < R; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < R; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
          for (int j = i; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    } else {
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double a[R], b[R];
#pragma unroll
        for (int i = 0; i < R; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < R; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
          for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  double* Cz = C + (long long)blockIdx.z * split_stride;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int r = m0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      int c = n0 + tx + 16 * j;
      if (c < N) Cz[(long long)r * ldc + c] = acc[i][j];
    }
  }
}

int gram_tile() { return 32; }

// Returns the number of split-K partial products written (nsplit after rounding the
// K chunk up to a multiple of BK): the partials a reduction must read.
int launch_gemm_nt_f64(const double* A, long long lda, const double* B, long long ldb, double* C,
                       long long ldc, long long split_stride, int M, int N, long long K,
                       int nsplit, int upper_only, cudaStream_t s) {
  if (nsplit < 1) nsplit = 1;
  long long kchunk = (K + nsplit - 1) / nsplit;
  kchunk = (kchunk + BK - 1) / BK * BK;
  nsplit = (int)((K + kchunk - 1) / kchunk);
  if (nsplit < 1) nsplit = 1;
  if (upper_only) {   // symmetric Grams: the upper triangle of 32 x 32 tiles
    constexpr int T = 32;
    const int nt = (M + T - 1) / T;
    gemm_nt_f64_kernel<T><<<dim3(nt * (nt + 1) / 2, 1, nsplit), 256, 0, s>>>(A, lda, B, ldb, C, ldc,
                                                                            split_stride, M, N, K, kchunk, 1);
  } else {
    gemm_nt_f64_kernel<BM><<<dim3((N + BN - 1) / BN, (M + BM - 1) / BM, nsplit), 256, 0, s>>>(
        A, lda, B, ldb, C, ldc, split_stride, M, N, K, kchunk, 0);
  }
  ++g_launches;
  return nsplit;
}

// Batched small FP64 products for the Newton-Schulz re-orthonormalisation in the
// eigen-solver: C_b = A_b . op(B_b), op(B) = B^T (B_N = false: B rows are K-contiguous)
// or B (B_N = true: B[k][j], j contiguous).  64 x 64 tiles, 4 x 4 per thread.
template <bool B_N>
__global__ void __launch_bounds__(256) gemm_small_f64_kernel(
    const double* __restrict__ A, long long lda, const double* __restrict__ B, long long ldb,
    double* __restrict__ C, long long ldc, int M, int N, int K, long long bsa, long long bsb,
    long long bsc) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  A += blockIdx.z * bsa;
  B += blockIdx.z * bsb;
  C += blockIdx.z * bsc;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int k = k0 + lk + u;
      int ra = m0 + lr;
      As[lk + u][lr] = (ra < M && k < K) ? A[(long long)ra * lda + k] : 0.0;
      if (!B_N) {
        int rb = n0 + lr;
        Bs[lk + u][lr] = (rb < N && k < K) ? B[(long long)rb * ldb + k] : 0.0;
      } else {
        int kk = tid >> 4, col = (tid & 15) * 4 + u;
        int kb = k0 + kk;
        Bs[kk][col] = (kb < K && n0 + col < N) ? B[(long long)kb * ldb + n0 + col] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = m0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = n0 + tx + 16 * j;
      if (c < N) C[(long long)r * ldc + c] = acc[i][j];
    }
  }
}

void launch_gemm_nn_f64(const double* A, long long lda, const double* B, long long ldb, double* C,
                        long long ldc, int M, int N, int K, int batch, long long bsa, long long bsb,
                        long long bsc, cudaStream_t s) {
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  gemm_small_f64_kernel<true><<<grid, 256, 0, s>>>(A, lda, B, ldb, C, ldc, M, N, K, bsa, bsb, bsc);
  ++g_launches;
}

void launch_gemm_nt_f64_batched(const double* A, long long lda, const double* B, long long ldb,
                                double* C, long long ldc, int M, int N, int K, int batch,
                                long long bsa, long long bsb, long long bsc, cudaStream_t s) {
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  gemm_small_f64_kernel<false><<<grid, 256, 0, s>>>(A, lda, B, ldb, C, ldc, M, N, K, bsa, bsb, bsc);
  ++g_launches;
}

// G[i][j] = sum_z parts[z][min(i,j)][max(i,j)]  (exactly symmetric)
__global__ void reduce_sym_kernel(const double* __restrict__ parts, int nsplit, int m,
                                  double* __restrict__ G) {
  long long total = (long long)m * m;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / m), j = (int)(e % m);
    int lo = i < j ? i : j, hi = i < j ? j : i;
    double acc = 0.0;
    for (int z = 0; z < nsplit; ++z) acc += parts[(long long)z * total + (long long)lo * m + hi];
    G[e] = acc;
  }
}

void launch_reduce_sym(const double* parts, int nsplit, int m, double* G, cudaStream_t s) {
  long long total = (long long)m * m;
  int blocks = (int)((total + 255) / 256);
  reduce_sym_kernel<<<blocks, 256, 0, s>>>(parts, nsplit, m, G);
  ++g_launches;
}

// A_{(f^ + f~ chi),(g^ + g~ chi)} = sum_{rho, eta} S^_{(f^ rho),(g^ eta)} S~_{(f~ rho),(g~ eta)}
// (Sec. 3.2, last step; S rows are (n_j, current) with n_j the slow index).
// Computed for the upper triangle and mirrored, so A is exactly symmetric.
__global__ void assemble_a_kernel(const double* __restrict__ sh, const double* __restrict__ sc,
                                  int chi, int chc, double* __restrict__ A) {
  int n = chi * chi;
  int m = chi * chc;
  long long total = (long long)n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    if (i > j) continue;
    int fh = i % chi, fc = i / chi, gh = j % chi, gc = j / chi;
    const double* shr = sh + (long long)(fh * chc) * m + gh * chc;
    const double* scr = sc + (long long)(fc * chc) * m + gc * chc;
    double acc = 0.0;
    for (int rho = 0; rho < chc; ++rho)
      for (int eta = 0; eta < chc; ++eta)
        acc = fma(shr[(long long)rho * m + eta], scr[(long long)rho * m + eta], acc);
    A[(long long)i * n + j] = acc;
    A[(long long)j * n + i] = acc;
  }
}

void launch_assemble_a(const double* s_hat, const double* s_chk, int chi_j, int chi_c, double* A,
                       cudaStream_t s) {
  long long total = (long long)chi_j * chi_j * chi_j * chi_j;
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  assemble_a_kernel<<<(unsigned)blocks, 256, 0, s>>>(s_hat, s_chk, chi_j, chi_c, A);
  ++g_launches;
}

// FP64 FMA throughput probe: every thread runs eight independent chains
// x <- x * a + b (|a| < 1, so the values stay bounded), `iters` steps each, and
// writes one sum so that the chains are not removed.  2 flops per FMA.
__global__ void __launch_bounds__(256) dfma_rate_kernel(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double sum = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) sum += x[k];
  if (threadIdx.x == 0) out[blockIdx.x] = sum;
}

int measure_fp64_rate(double* tflops) {
  const int sms = sm_count(), blocks = 8 * sms, threads = 256, iters = 1 << 15;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks) != cudaSuccess) {
    cudaGetLastError();
    return -2;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 0.0f;
  for (int rep = 0; rep < 3; ++rep) {   // the first launch warms up (clocks, module load)
    cudaEventRecord(e0, 0);
    dfma_rate_kernel<<<blocks, threads>>>(out, iters, 0.9999999, 1e-7);
    ++g_launches;
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || best <= 0.0f) return -3;
  *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
  return 0;
}

}  // namespace hotrg
