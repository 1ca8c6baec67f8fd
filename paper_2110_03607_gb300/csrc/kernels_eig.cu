// Batched FP64 one-sided (Hestenes) Jacobi eigen-solver for the symmetric
// PSD environment matrices A^(j), A'^(j) (Sec. 4.2.5, Eqs. SVD_N / SVD_P),
// and the choice / truncation / sign gauge of the isometries (Secs. 2,
// 4.2.6-4.2.8).
//
// One-sided Jacobi: W = A V is orthogonalised column pair by column pair by
// plane rotations applied to W and V; at convergence the columns of W are
// mutually orthogonal, so V diagonalises A^T A = A^2 and, A being PSD,
// A v_i = lambda_i v_i with lambda_i = ||w_i||.  Pairs follow the round-robin
// ordering (n/2 disjoint pairs per round, n-1 rounds per sweep), so every
// pair of a round -- over all matrices of the batch -- runs in parallel on
// its own warp; rounds are separated by a grid-wide barrier of a cooperative
// launch.  A pair whose inner product is exactly 0 is never rotated, which
// keeps an exact Z2 block pattern of A exact.
//
// Stopping rule: a sweep counts only the rotations of pairs in which a column's
// squared norm exceeds (4 n eps)^2 times the largest squared column norm at the
// start (about lambda_1^2): the solver stops after a sweep that rotates no such
// pair.  Pairs of two columns below that floor -- the near-null space of A, whose
// columns are rounding noise of order n eps lambda_1 -- are still rotated as
// before, but their mutual orthogonalisation no longer keeps the sweeps going:
// every column above the floor is then orthogonal to every other column to the
// rotation tolerance, so its vector is an eigenvector as before, and the columns
// below it span the rest of the space (V stays orthogonal).
#include <cooperative_groups.h>

#include "hotrg_internal.cuh"
#include "../../include/hotrg.h"

namespace cg = cooperative_groups;

namespace hotrg {

__device__ __forceinline__ int rr_slot(int i, int r, int mp) {
  // circle method: player 0 fixed, the others rotate by r (0 <= i - 1 + r < 2 (mp - 1), so
  // one conditional subtraction replaces the modulo)
  if (i == 0) return 0;
  int x = i - 1 + r;
  if (x >= mp - 1) x -= mp - 1;
  return 1 + x;
}

// NPL = ceil(n / 32): column entries held per lane
template <int NPL>
__global__ void __launch_bounds__(256) jacobi_onesided_kernel(double* W, double* V,
                                                               const double* __restrict__ A, int n,
                                                               int nmat, int max_sweeps,
                                                               int* counters, unsigned long long* colmax,
                                                               int* sweeps_out, DevState* st) {
  cg::grid_group grid = cg::this_grid();
  const long long nn = (long long)n * n;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gthreads = (long long)gridDim.x * blockDim.x;
  // A == nullptr: W and V already hold a starting point (W = A V, V orthogonal)
  if (A) {
    for (long long e = gtid; e < (long long)nmat * nn; e += gthreads) {
      long long r = e % nn;
      int i = (int)(r / n), j = (int)(r % n);
      __stcg(W + e, A[e]);                // A symmetric: row i = column i
      __stcg(V + e, i == j ? 1.0 : 0.0);
    }
  }
  if (gtid < 3 * nmat) counters[gtid] = 0;
  if (gtid < nmat) colmax[gtid] = 0ull;
  grid.sync();

  const int mp = n + (n & 1);
  const int npairs = mp / 2;
  const int rounds = mp - 1;
  const int lane = threadIdx.x & 31;
  // consecutive tasks go to different blocks (SMs), spreading the FP64 work
  const int gw = (int)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const int nw = (int)(gthreads >> 5);
  const int ntasks = nmat * npairs;
  // largest squared column norm of every matrix (non-negative doubles order like their
  // bit patterns, so an integer maximum is exact and independent of the order)
  for (int task = gw; task < nmat * n; task += nw) {
    const int mat = task / n, col = task % n;
    const double* w = W + mat * nn + (long long)col * n;
    double a = 0.0;
    for (int i = lane; i < n; i += 32) {
      const double x = __ldcg(w + i);
      a = fma(x, x, a);
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0 && a > 0.0) atomicMax(colmax + mat, (unsigned long long)__double_as_longlong(a));
  }
  grid.sync();
  // fixed for the whole solve: read once into shared memory (nmat <= 16)
  __shared__ double s_amax[16];
  if ((int)threadIdx.x < nmat) s_amax[threadIdx.x] = __longlong_as_double((long long)__ldcg(colmax + threadIdx.x));
  __syncthreads();
  // the computed inner product carries rounding of order n eps sqrt(a b): a
  // tolerance below that level would keep rotating rounding noise forever.  A pair
  // is rotated only if |g| > tol max(a, b), not tol sqrt(a b): the rotation it would
  // apply to V is g / (a - b), below tol either way, but a column at rounding level
  // (a near-null direction of A) carries noise of order eps times the large column it
  // was last rotated against, and the relative test would rotate that pair forever.
  // Columns with a squared norm below 1e-280 are left alone: their squares and products
  // are subnormal, tol max(a, b) underflows to 0, and any nonzero g would rotate them
  // forever (the environments of a trace-normalised tensor have lambda_1 >> 1e-140)
  const double tol = 4.0 * (double)n * 2.220446049250313e-16;

  int sweep = 1;
  bool converged = false;
  for (; sweep <= max_sweeps; ++sweep) {
    int* cur = counters + (sweep % 3) * nmat;
    if (blockIdx.x == 0 && (int)threadIdx.x < nmat) counters[((sweep + 1) % 3) * nmat + threadIdx.x] = 0;
    for (int r = 0; r < rounds; ++r) {
      for (int task = gw; task < ntasks; task += nw) {
        int mat = task / npairs, k = task % npairs;
        int p = rr_slot(k, r, mp), q = rr_slot(mp - 1 - k, r, mp);
        if (p >= n || q >= n) continue;
        if (p > q) { int t = p; p = q; q = t; }
        double* wp = W + mat * nn + (long long)p * n;
        double* wq = W + mat * nn + (long long)q * n;
        double* vp = V + mat * nn + (long long)p * n;
        double* vq = V + mat * nn + (long long)q * n;
        // up to 256 rows the V columns are loaded with the W columns (independent loads,
        // one L2 round trip on the pair's path instead of two); used only if it rotates
        constexpr bool kVreg = NPL <= 8;
        double vxs[kVreg ? NPL : 1], vys[kVreg ? NPL : 1];
        double a = 0.0, b = 0.0, g = 0.0;
        double xs[NPL], ys[NPL];
#pragma unroll
        for (int u = 0; u < NPL; ++u) {
          int i = lane + 32 * u;
          xs[u] = i < n ? __ldcg(wp + i) : 0.0;
          ys[u] = i < n ? __ldcg(wq + i) : 0.0;
          if constexpr (kVreg) {
            vxs[u] = i < n ? __ldcg(vp + i) : 0.0;
            vys[u] = i < n ? __ldcg(vq + i) : 0.0;
          }
        }
#pragma unroll
        for (int u = 0; u < NPL; ++u) {
          a = fma(xs[u], xs[u], a);
          b = fma(ys[u], ys[u], b);
          g = fma(xs[u], ys[u], g);
        }
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        const double big = fmax(a, b);
        bool rot = (g != 0.0) && big > 1e-280 && (fabs(g) > tol * big);
        if (!rot) continue;
        const bool counts = big > tol * tol * s_amax[mat];
        double zeta = (b - a) / (2.0 * g);
        double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = c * t;
#pragma unroll
        for (int u = 0; u < NPL; ++u) {
          int i = lane + 32 * u;
          if (i < n) {
            __stcg(wp + i, c * xs[u] - s * ys[u]);
            __stcg(wq + i, s * xs[u] + c * ys[u]);
          }
        }
        if constexpr (kVreg) {
#pragma unroll
          for (int u = 0; u < NPL; ++u) {
            int i = lane + 32 * u;
            if (i < n) {
              __stcg(vp + i, c * vxs[u] - s * vys[u]);
              __stcg(vq + i, s * vxs[u] + c * vys[u]);
            }
          }
        } else {
          for (int i = lane; i < n; i += 32) {
            double x = __ldcg(vp + i), y = __ldcg(vq + i);
            __stcg(vp + i, c * x - s * y);
            __stcg(vq + i, s * x + c * y);
          }
        }
        if (lane == 0 && counts) atomicAdd(cur + mat, 1);
      }
      grid.sync();
    }
    int total = 0;
    for (int m = 0; m < nmat; ++m) total += __ldcg(cur + m);
    if (total == 0) {
      converged = true;
      break;
    }
  }
  if (gtid == 0) {
    for (int m = 0; m < nmat; ++m) sweeps_out[m] = sweep;
    if (!converged && st->status == 0) st->status = HOTRG_ENOTCONV;
  }
}

template <int NPL>
static int launch_jacobi_t(double* W, double* V, const double* A, int n, int nmat, int max_sweeps,
                           int* counters, unsigned long long* colmax, int* sweeps_out, DevState* st,
                           cudaStream_t s) {
  // resident CTAs per SM, queried once per device
  static std::atomic<int> per_cache[kMaxDevices];
  int dev = 0;
  cudaGetDevice(&dev);
  int per = (dev >= 0 && dev < kMaxDevices) ? per_cache[dev].load(std::memory_order_relaxed) : 0;
  if (per < 1) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi_onesided_kernel<NPL>, 256, 0) !=
            cudaSuccess ||
        per < 1) {
      cudaGetLastError();
      per = 1;
    }
    if (dev >= 0 && dev < kMaxDevices) per_cache[dev].store(per, std::memory_order_relaxed);
  }
  const int s_sms = sm_count(), s_per_sm = per;
  int mp = n + (n & 1);
  int tasks = nmat * (mp / 2);
  // one block per SM (up to the task count): tasks are dealt round-robin over blocks
  int blocks = tasks < s_sms ? tasks : s_sms;
  if (blocks > s_sms * s_per_sm) blocks = s_sms * s_per_sm;
  if (blocks < 1) blocks = 1;
  void* args[] = {&W, &V, &A, &n, &nmat, &max_sweeps, &counters, &colmax, &sweeps_out, &st};
  cudaError_t e = cudaLaunchCooperativeKernel((void*)jacobi_onesided_kernel<NPL>, dim3(blocks),
                                              dim3(256), args, 0, s);
  ++g_launches;
  return e == cudaSuccess ? 0 : -1;
}

int launch_jacobi(double* W, double* V, const double* A, int n, int nmat, int max_sweeps,
                  int* counters, unsigned long long* colmax, int* sweeps_out, DevState* st,
                  cudaStream_t s) {
  if (nmat > 16) return -1;
  const int npl = (n + 31) / 32;
#define HOTRG_JAC(P) return launch_jacobi_t<P>(W, V, A, n, nmat, max_sweeps, counters, colmax, sweeps_out, st, s)
  if (npl <= 1) HOTRG_JAC(1);
  if (npl <= 2) HOTRG_JAC(2);
  if (npl <= 4) HOTRG_JAC(4);
  if (npl <= 8) HOTRG_JAC(8);
  if (npl <= 16) HOTRG_JAC(16);
  if (npl <= 32) HOTRG_JAC(32);
#undef HOTRG_JAC
  return -1;
}

// ---------------------------------------------------------------------------
// FP32 warm start: block one-sided Jacobi.  The n columns of W = A V are cut
// into nb blocks of b; an outer round pairs the blocks round-robin and one CTA
// per block pair loads its 2b columns of W and V into shared memory, runs one
// inner sweep of one-sided Jacobi over them (2b-1 inner rounds of b disjoint
// pairs, separated by __syncthreads), and writes them back.  Outer rounds are
// separated by a grid barrier of a cooperative launch, so a sweep costs nb-1
// grid barriers instead of n-1.  Its vectors only seed the FP64 sweeps, which
// restore full accuracy; it stops when an outer sweep rotates nothing, or after
// max_sweeps, without raising an error.
// ---------------------------------------------------------------------------
template <int NPL>
__global__ void __launch_bounds__(1024) jacobi32_block_kernel(const double* __restrict__ A, float* W,
                                                              float* V, int n, int b, int nb,
                                                              int nmat, int max_sweeps, int* counters) {
  extern __shared__ float jsm[];
  __shared__ int s_rot;
  cg::grid_group grid = cg::this_grid();
  const long long nn = (long long)n * n;
  const int kpairs = nb / 2;
  const int mat = blockIdx.x / kpairs, kp = blockIdx.x % kpairs;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gthreads = (long long)gridDim.x * blockDim.x;
  for (long long e = gtid; e < (long long)nmat * nn; e += gthreads) {
    long long r = e % nn;
    W[e] = (float)A[e];
    V[e] = (r / n == r % n) ? 1.0f : 0.0f;
  }
  if (gtid < 3) counters[gtid] = 0;
  grid.sync();
  float* Wm = W + mat * nn;
  float* Vm = V + mat * nn;
  float* sw = jsm;                          // [2b][n]
  float* sv = jsm + (long long)2 * b * n;   // [2b][n]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float tol = 4.0f * (float)n * 1.1920929e-7f;
  const int m2 = 2 * b;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int* cur = counters + (sweep % 3);
    if (gtid == 0) counters[(sweep + 1) % 3] = 0;
    for (int r = 0; r < nb - 1; ++r) {
      const int bi = rr_slot(kp, r, nb), bj = rr_slot(nb - 1 - kp, r, nb);
      // local column c < b is block bi's column, c >= b block bj's
      for (long long e = threadIdx.x; e < (long long)m2 * n; e += blockDim.x) {
        int c = (int)(e / n), i = (int)(e % n);
        int gc = (c < b ? bi * b + c : bj * b + (c - b));
        bool in = gc < n;
        sw[e] = in ? Wm[(long long)gc * n + i] : 0.0f;
        sv[e] = in ? Vm[(long long)gc * n + i] : 0.0f;
      }
      if (threadIdx.x == 0) s_rot = 0;
      __syncthreads();
      for (int ir = 0; ir < m2 - 1; ++ir) {
        for (int k = warp; k < b; k += nw) {
          int p = rr_slot(k, ir, m2), q = rr_slot(m2 - 1 - k, ir, m2);
          if (p > q) { int t = p; p = q; q = t; }
          float* wp = sw + (long long)p * n;
          float* wq = sw + (long long)q * n;
          float xs[NPL], ys[NPL];
          float a = 0.f, bb = 0.f, g = 0.f;
#pragma unroll
          for (int u = 0; u < NPL; ++u) {
            int i = lane + 32 * u;
            float x = i < n ? wp[i] : 0.f, y = i < n ? wq[i] : 0.f;
            xs[u] = x;
            ys[u] = y;
            a = fmaf(x, x, a);
            bb = fmaf(y, y, bb);
            g = fmaf(x, y, g);
          }
          for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            bb += __shfl_xor_sync(0xffffffffu, bb, o);
            g += __shfl_xor_sync(0xffffffffu, g, o);
          }
          if (g == 0.f || !(fabsf(g) > tol * sqrtf(a * bb))) continue;
          float zeta = (bb - a) / (2.f * g);
          float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          float c = 1.f / sqrtf(1.f + t * t), sn = c * t;
          float* vp = sv + (long long)p * n;
          float* vq = sv + (long long)q * n;
#pragma unroll
          for (int u = 0; u < NPL; ++u) {
            int i = lane + 32 * u;
            if (i < n) {
              wp[i] = c * xs[u] - sn * ys[u];
              wq[i] = sn * xs[u] + c * ys[u];
              float x = vp[i], y = vq[i];
              vp[i] = c * x - sn * y;
              vq[i] = sn * x + c * y;
            }
          }
          if (lane == 0) atomicAdd(&s_rot, 1);
        }
        __syncthreads();
      }
      for (long long e = threadIdx.x; e < (long long)m2 * n; e += blockDim.x) {
        int c = (int)(e / n), i = (int)(e % n);
        int gc = (c < b ? bi * b + c : bj * b + (c - b));
        if (gc < n) {
          Wm[(long long)gc * n + i] = sw[e];
          Vm[(long long)gc * n + i] = sv[e];
        }
      }
      if (threadIdx.x == 0 && s_rot) atomicAdd(cur, s_rot);
      grid.sync();
    }
    if (__ldcg(cur) == 0) break;
  }
}

// FP32 warm start for n <= 170: one CTA per matrix holds all of W and V in shared
// memory (2 n^2 floats) and runs the round-robin sweeps of one-sided Jacobi with a
// __syncthreads between rounds -- no grid barrier.  Same rotation test and stopping
// rule as the block version below.
template <int NPL>
__global__ void __launch_bounds__(1024, 1) jacobi32_smem_kernel(const double* __restrict__ A, float* W, float* V,
                                                                int n, int max_sweeps) {
  extern __shared__ float jsm[];
  __shared__ int s_rot;
  const long long nn = (long long)n * n;
  float* sw = jsm;
  float* sv = jsm + nn;
  const double* Am = A + blockIdx.x * nn;
  for (int e = threadIdx.x; e < (int)nn; e += blockDim.x) {
    sw[e] = (float)Am[e];                       // A symmetric: row i = column i
    sv[e] = (e / n == e % n) ? 1.0f : 0.0f;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int mp = n + (n & 1), npairs = mp / 2, rounds = mp - 1;
  const float tol = 4.0f * (float)n * 1.1920929e-7f;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < rounds; ++r) {
      for (int k = warp; k < npairs; k += nw) {
        int p = rr_slot(k, r, mp), q = rr_slot(mp - 1 - k, r, mp);
        if (p >= n || q >= n) continue;
        if (p > q) { int t = p; p = q; q = t; }
        float* wp = sw + (long long)p * n;
        float* wq = sw + (long long)q * n;
        float xs[NPL], ys[NPL];
        float a = 0.f, bb = 0.f, g = 0.f;
#pragma unroll
        for (int u = 0; u < NPL; ++u) {
          int i = lane + 32 * u;
          float x = i < n ? wp[i] : 0.f, y = i < n ? wq[i] : 0.f;
          xs[u] = x;
          ys[u] = y;
          a = fmaf(x, x, a);
          bb = fmaf(y, y, bb);
          g = fmaf(x, y, g);
        }
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          bb += __shfl_xor_sync(0xffffffffu, bb, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        if (g == 0.f || !(fabsf(g) > tol * sqrtf(a * bb))) continue;
        float zeta = (bb - a) / (2.f * g);
        float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        float c = 1.f / sqrtf(1.f + t * t), sn = c * t;
        float* vp = sv + (long long)p * n;
        float* vq = sv + (long long)q * n;
#pragma unroll
        for (int u = 0; u < NPL; ++u) {
          int i = lane + 32 * u;
          if (i < n) {
            wp[i] = c * xs[u] - sn * ys[u];
            wq[i] = sn * xs[u] + c * ys[u];
            float x = vp[i], y = vq[i];
            vp[i] = c * x - sn * y;
            vq[i] = sn * x + c * y;
          }
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (rot == 0) break;
  }
  float* Wm = W + blockIdx.x * nn;
  float* Vm = V + blockIdx.x * nn;
  for (int e = threadIdx.x; e < (int)nn; e += blockDim.x) {
    Wm[e] = sw[e];
    Vm[e] = sv[e];
  }
}

// Block size b: four blocks (three outer rounds, one grid barrier each, per sweep) when
// two blocks of W and V fit in 200 KB of shared memory, else b = 32 (or less) and
// nb = ceil(n / b) rounded up to even.
int launch_jacobi32_block(const double* A, float* W32, float* V32, int n, int nmat, int max_sweeps,
                          int* counters, cudaStream_t s) {
  {
    const size_t smem1 = (size_t)2 * n * n * sizeof(float);
    const int npl1 = (n + 31) / 32;
    if (smem1 <= 227 * 1024 && npl1 <= 8) {
      void* k1 = npl1 <= 2 ? (void*)jacobi32_smem_kernel<2>
               : npl1 <= 4 ? (void*)jacobi32_smem_kernel<4> : (void*)jacobi32_smem_kernel<8>;
      if (cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1) != cudaSuccess)
        return -1;
      void* args1[] = {&A, &W32, &V32, &n, &max_sweeps};
      const cudaError_t e1 = cudaLaunchKernel(k1, dim3(nmat), dim3(1024), args1, smem1, s);
      ++g_launches;
      return e1 == cudaSuccess ? 0 : -1;
    }
  }
  int b = (n + 3) / 4;
  if (b > 64 || (size_t)4 * b * n * sizeof(float) > 200 * 1024) {
    b = 32;
    while (b > 4 && (size_t)4 * b * n * sizeof(float) > 200 * 1024) b /= 2;
  }
  int nb = (n + b - 1) / b;
  if (nb & 1) ++nb;
  if (nb < 2) nb = 2;
  size_t smem = (size_t)4 * b * n * sizeof(float);
  if (smem > 200 * 1024) return -1;
  int npl = (n + 31) / 32;
  void* kern = nullptr;
  if (npl <= 2) kern = (void*)jacobi32_block_kernel<2>;
  else if (npl <= 4) kern = (void*)jacobi32_block_kernel<4>;
  else if (npl <= 8) kern = (void*)jacobi32_block_kernel<8>;
  else if (npl <= 16) kern = (void*)jacobi32_block_kernel<16>;
  else return -1;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -1;
  int blocks = nmat * (nb / 2);
  void* args[] = {&A, &W32, &V32, &n, &b, &nb, &nmat, &max_sweeps, &counters};
  cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(1024), args, smem, s);
  ++g_launches;
  return e == cudaSuccess ? 0 : -1;
}

// Q = V32 in FP64, and 0.5 (3 I - G) for the Newton-Schulz step Q <- Q (3I - Q^T Q) / 2
__global__ void widen_f32_kernel(const float* __restrict__ in, double* __restrict__ out, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (double)in[e];
}

__global__ void ns_coeff_kernel(double* G, int n, long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e % ((long long)n * n);
    int i = (int)(r / n), j = (int)(r % n);
    G[e] = (i == j ? 1.5 : 0.0) - 0.5 * G[e];
  }
}

void launch_widen_f32(const float* in, double* out, long long n, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  widen_f32_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, out, n);
  ++g_launches;
}

void launch_ns_coeff(double* G, int n, int nmat, cudaStream_t s) {
  long long total = (long long)nmat * n * n;
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  ns_coeff_kernel<<<(unsigned)blocks, 256, 0, s>>>(G, n, total);
  ++g_launches;
}

// ---------------------------------------------------------------------------
// Choice, truncation and sign gauge for one transverse leg.
// Matrices 2*leg (A^(j)) and 2*leg+1 (A'^(j)) of the Jacobi batch are used.
// Orders the eigenpairs by lambda descending; values within 1e-12 lambda_1 of
// their predecessor form a tie group ordered by pivot index (the lowest row
// whose magnitude is within 1e-6 of the column maximum).  epsilon = sum of the
// eigenvalues after the first nnew; U^(j) is taken if epsilon < epsilon' -
// 1e-10 max(lambda_1, lambda'_1), else U'^(j); each kept column is flipped so
// that its pivot entry is positive.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) select_kernel(const double* __restrict__ W,
                                                     const double* __restrict__ V, int n,
                                                     int leg_index, int nnew, double* lam_sorted,
                                                     double* U64, float* U32, LegResult* res,
                                                     const int* sweeps, int* rank_out) {
  extern __shared__ double sm[];
  double* lam = sm;                         // [2][n]
  int* piv = (int*)(lam + 2 * n);           // [2][n]
  int* sgn = piv + 2 * n;                   // [2][n]
  int* order = sgn + 2 * n;                 // [2][n]
  __shared__ double s_eps[2];
  __shared__ int s_choice;
  const long long nn = (long long)n * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int side = 0; side < 2; ++side) {
    const double* Wm = W + (long long)(2 * leg_index + side) * nn;
    const double* Vm = V + (long long)(2 * leg_index + side) * nn;
    for (int i = warp; i < n; i += nwarps) {
      double s2 = 0.0, vmax = 0.0;
      for (int k = lane; k < n; k += 32) {
        double w = Wm[(long long)i * n + k];
        s2 = fma(w, w, s2);
        vmax = fmax(vmax, fabs(Vm[(long long)i * n + k]));
      }
      for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      }
      int first = n;
      for (int k0 = 0; k0 < n && first == n; k0 += 32) {
        int k = k0 + lane;
        bool hit = k < n && fabs(Vm[(long long)i * n + k]) >= (1.0 - 1e-6) * vmax;
        unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m) first = k0 + __ffs(m) - 1;
      }
      if (first >= n) first = 0;   // no entry found (a NaN column): stay in range; the trace reports it
      if (lane == 0) {
        lam[side * n + i] = sqrt(s2);
        piv[side * n + i] = first;
        sgn[side * n + i] = Vm[(long long)i * n + first] < 0.0 ? -1 : 1;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * n; e += blockDim.x) {
    int side = e / n, i = e % n;
    const double* l = lam + side * n;
    // a NaN ranks below every number, so that the ranks stay a permutation
    const double li = isnan(l[i]) ? -1.0 : l[i];
    int rank = 0;
    for (int k = 0; k < n; ++k) {
      const double lk = isnan(l[k]) ? -1.0 : l[k];
      rank += (lk > li) || (lk == li && k < i);
    }
    order[side * n + rank] = i;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    int side = threadIdx.x;
    const double* l = lam + side * n;
    int* ord = order + side * n;
    const int* pv = piv + side * n;
    double tol = 1e-12 * l[ord[0]];
    int g0 = 0;
    for (int r = 1; r <= n; ++r) {
      bool brk = (r == n) || (l[ord[r - 1]] - l[ord[r]] > tol);
      if (brk) {
        // insertion sort of ord[g0 .. r-1] by pivot index
        for (int a = g0 + 1; a < r; ++a) {
          int key = ord[a];
          int b = a - 1;
          while (b >= g0 && pv[ord[b]] > pv[key]) {
            ord[b + 1] = ord[b];
            --b;
          }
          ord[b + 1] = key;
        }
        g0 = r;
      }
    }
    double eps = 0.0;
    for (int r = nnew; r < n; ++r) eps += l[ord[r]];
    s_eps[side] = eps;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double l1a = lam[order[0]], l1b = lam[n + order[n]];
    double tol = 1e-10 * fmax(l1a, l1b);
    int prime = !(s_eps[0] < s_eps[1] - tol) ? 1 : 0;
    s_choice = prime;
    const double* lc = lam + prime * n;
    const int* oc = order + prime * n;
    res->eps[0] = s_eps[0];
    res->eps[1] = s_eps[1];
    res->lam1[0] = l1a;
    res->lam1[1] = l1b;
    res->chose_prime = prime;
    res->sweeps[0] = sweeps ? sweeps[0] : 0;
    res->sweeps[1] = sweeps ? sweeps[1] : 0;
    res->gap = (nnew < n && lc[oc[0]] > 0.0) ? (lc[oc[nnew - 1]] - lc[oc[nnew]]) / lc[oc[0]] : 1e300;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * n; e += blockDim.x) {
    int side = e / n, r = e % n;
    lam_sorted[e] = lam[side * n + order[side * n + r]];
  }
  const int side = s_choice;
  if (rank_out)   // rank of every eigenvector of the chosen side in the sorted order
    for (int r = threadIdx.x; r < n; r += blockDim.x) rank_out[order[side * n + r]] = r;
  const double* Vm = V + (long long)(2 * leg_index + side) * nn;
  for (int e = threadIdx.x; e < n * nnew; e += blockDim.x) {
    int row = e / nnew, col = e % nnew;
    int src = order[side * n + col];
    double v = Vm[(long long)src * n + row] * (double)sgn[side * n + src];
    U64[e] = v;
    U32[e] = (float)v;
  }
}

void launch_select(const double* W, const double* V, int n, int leg_index, int nnew,
                   double* lam_sorted, double* U64, float* U32, LegResult* res,
                   const int* sweeps, cudaStream_t s, int* rank_out) {
  size_t smem = (size_t)2 * n * sizeof(double) + (size_t)6 * n * sizeof(int);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  select_kernel<<<1, 512, smem, s>>>(W, V, n, leg_index, nnew, lam_sorted, U64, U32, res, sweeps, rank_out);
  ++g_launches;
}

}  // namespace hotrg
