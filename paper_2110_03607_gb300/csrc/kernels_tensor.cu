// Elementwise and reduction kernels around the step: initial Ising tensor
// (Sec. 2, Eq. 2.4), leg permutations (the renaming of Sec. 3.1.3 and the
// gathers of the environment Grams), BF16 splitting of the contraction
// operands, the Y matrix / trace / Gu-Wen ratio (Sec. 4.1.2, Sec. 4.2.11)
// and the normalisation with ln Z bookkeeping (Sec. 4.1.1, Secs. 4.2.14-16).
#include "hotrg_internal.cuh"
#include "../../include/hotrg.h"

namespace hotrg {

std::atomic<long long> g_launches{0};

int sm_count() {
  static std::atomic<int> cache[kMaxDevices];   // zero until queried
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  int v = (dev >= 0 && dev < kMaxDevices) ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    cudaGetLastError();
    v = 1;
  }
  if (dev >= 0 && dev < kMaxDevices) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// T0 in the slot layout rows (x_0 .. x_{d-1}) x cols (x_0' .. x_{d-1}').
// Every leg carries X_{s j}: X_{s 0} = sqrt(cosh b), X_{s 1} = sigma_s sqrt(sinh b)
// (X = U sqrt(Lambda), U = [[1,1],[1,-1]]/sqrt 2, Lambda = diag(2cosh b, 2sinh b)),
// and the site weight is V_s = exp(b h sigma_s), sigma_0 = +1, sigma_1 = -1.
__global__ void init_ising_kernel(double* T, int d, double beta, double h) {
  int n = 1 << (2 * d);
  double x0 = sqrt(cosh(beta));
  double x1 = sqrt(sinh(beta));
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    int ones = __popc(e);
    double acc = 0.0;
    for (int s = 0; s < 2; ++s) {
      double sigma = s == 0 ? 1.0 : -1.0;
      double prod = exp(beta * h * sigma);
      for (int leg = 0; leg < 2 * d; ++leg) {
        int bit = (e >> leg) & 1;
        prod *= bit ? sigma * x1 : x0;
      }
      acc += prod;
    }
    (void)ones;
    T[e] = acc;
  }
}

void launch_init_ising(double* T, int d, double beta, double h, cudaStream_t s) {
  init_ising_kernel<<<1, 256, 0, s>>>(T, d, beta, h);
  ++g_launches;
}

// out (C order over out_size) = scale * in[sum idx_k in_stride_k]
struct PermArgs {
  int ndim;
  unsigned size[kMaxDims];
  long long in_stride[kMaxDims];
  unsigned long long total;
};

__global__ void permute_kernel(const double* __restrict__ in, double* __restrict__ out,
                               PermArgs a, double scale) {
  unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long o = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; o < a.total;
       o += stride) {
    unsigned long long r = o;
    long long off = 0;
    for (int k = a.ndim - 1; k >= 0; --k) {
      unsigned sz = a.size[k];
      unsigned long long q = r / sz;
      unsigned idx = (unsigned)(r - q * sz);
      r = q;
      off += (long long)idx * a.in_stride[k];
    }
    out[o] = in[off] * scale;
  }
}

void launch_permute(const double* in, double* out, int ndim, const long long* out_size,
                    const long long* in_stride, double scale, cudaStream_t s) {
  PermArgs a;
  a.ndim = ndim;
  a.total = 1;
  for (int k = 0; k < ndim; ++k) {
    a.size[k] = (unsigned)out_size[k];
    a.in_stride[k] = in_stride[k];
    a.total *= (unsigned long long)out_size[k];
  }
  int threads = 256;
  long long blocks = (long long)((a.total + threads - 1) / threads);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  permute_kernel<<<(unsigned)blocks, threads, 0, s>>>(in, out, a, scale);
  ++g_launches;
}

// FP64 -> npieces pieces (BF16 or TF32): p0 = rnd(x), p1 = rnd(x - p0), p2 = rnd(x - p0 - p1),
// with x = in (+ in2, the same layout, when given).
__global__ void split_kernel(const double* __restrict__ in, const double* __restrict__ in2, long long rows,
                             long long cols, long long ld_in, void* __restrict__ out, long long ld_out,
                             long long piece_stride, int npieces, int pfmt) {
  long long total = rows * cols;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    long long r = e / cols, c = e - r * cols;
    double x = in2 ? in[r * ld_in + c] + in2[r * ld_in + c] : in[r * ld_in + c];
    store_pieces(out, r * ld_out + c, piece_stride, npieces, pfmt, x);
  }
}

void launch_split(const double* in, long long rows, long long cols, long long ld_in, void* out,
                  long long ld_out, long long piece_stride, int npieces, int pfmt, cudaStream_t s,
                  const double* in2) {
  long long total = rows * cols;
  long long blocks = (total + 255) / 256;
  if (blocks > 32LL * sm_count()) blocks = 32LL * sm_count();
  if (blocks < 1) blocks = 1;
  split_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, in2, rows, cols, ld_in, out, ld_out, piece_stride, npieces,
                                                pfmt);
  ++g_launches;
}

// Y_{c c'} = sum_n T_{(c, n), (c', n)} (Eq. Matrix_Y), one warp per (c, c').
__global__ void trace_y_kernel(const double* __restrict__ T, int chi_c, long long pn, double* Y) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= chi_c * chi_c) return;
  int c = warp / chi_c, cp = warp % chi_c;
  long long ld = (long long)chi_c * pn;
  double acc = 0.0;
  for (long long n = lane; n < pn; n += 32) acc += T[(c * pn + n) * ld + cp * pn + n];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) Y[warp] = acc;
}

void launch_trace_y(const double* Tn, int chi_c, long long pn, double* Y, cudaStream_t s) {
  int warps = chi_c * chi_c;
  int threads = 128;
  int blocks = (warps * 32 + threads - 1) / threads;
  trace_y_kernel<<<blocks, threads, 0, s>>>(Tn, chi_c, pn, Y);
  ++g_launches;
}

// Tr T = trace Y, X = (trace Y)^2 / trace(Y^2) (Eq. ratio_X); per-site form of
// the K recurrence (Eq. K_recurrence divided by 2^p):
//   kappa_p = kappa_{p-1} + ln Tr_{p-1} / 2^(p-1),   ln Z^(p)/V = kappa_p + ln Tr_p / 2^p.
__global__ void finish_step_kernel(const double* __restrict__ Y, int chi_c, DevState* st, int p,
                                   int first) {
  __shared__ double s_tr2[32];
  double tr2 = 0.0;
  for (int e = threadIdx.x; e < chi_c * chi_c; e += blockDim.x) {
    int c = e / chi_c, cp = e % chi_c;
    tr2 += Y[c * chi_c + cp] * Y[cp * chi_c + c];
  }
  for (int o = 16; o > 0; o >>= 1) tr2 += __shfl_xor_sync(0xffffffffu, tr2, o);
  if ((threadIdx.x & 31) == 0) s_tr2[threadIdx.x >> 5] = tr2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t2 += s_tr2[w];
    double tr = 0.0;
    for (int c = 0; c < chi_c; ++c) tr += Y[c * chi_c + c];
    if (!(tr > 0.0) || !isfinite(tr)) {
      if (st->status == 0) st->status = HOTRG_ENUMERIC;
      st->trace = tr;
      st->inv_trace = 1.0;
      return;
    }
    // p < 0: a step replayed from a captured graph takes its count from the device
    if (p < 0) p = st->p + 1;
    st->p = p;
    double ln_tr = log(tr);
    if (first) {
      st->kappa = 0.0;
      st->ln_z_site = ln_tr;
    } else {
      st->kappa = st->kappa + ldexp(st->ln_tr, -(p - 1));
      st->ln_z_site = st->kappa + ldexp(ln_tr, -p);
    }
    st->ln_tr = ln_tr;
    st->trace = tr;
    st->inv_trace = 1.0 / tr;
    st->gu_wen = tr * tr / t2;
  }
}

void launch_finish_step(double* Y, int chi_c, DevState* st, int p, int first, cudaStream_t s) {
  finish_step_kernel<<<1, 256, 0, s>>>(Y, chi_c, st, p, first);
  ++g_launches;
}

__global__ void scale_kernel(const double* __restrict__ in, double* __restrict__ out, long long n,
                             const DevState* st) {
  double f = st->inv_trace;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = in[i] * f;
}

void launch_scale(const double* in, double* out, long long n, const DevState* st, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  scale_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, out, n, st);
  ++g_launches;
}

}  // namespace hotrg
