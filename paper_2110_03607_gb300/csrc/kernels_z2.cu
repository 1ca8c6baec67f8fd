// Z2 (spin-flip) block structure of the bottleneck contraction at zero field.
//
// Every leg index carries a parity; the Ising tensor vanishes exactly on odd
// total parity (Sec. 2: column 0 of X is even, column 1 odd) and the isometries
// keep definite parities, so for a c'-slice of parity q the bottleneck of
// Eq. (BottleneckPart) splits into two dense blocks,
//   C_b[(c, n^) of parity b][(n', n~) of parity b ^ q]
//     = sum over (rho, n^') of parity b of T[.][.] B[.][.],   b = 0, 1,
// a quarter of the dense work.  These kernels gather the blocks into
// contiguous operands and scatter the products back into the dense layout
// (zeros elsewhere) that the non-prime chain reads.
#include "hotrg_internal.cuh"

namespace hotrg {

// dst[p][i][j] = piece p of src[rowmap[i] * ld + colmap[j]] (0 where colmap[j] < 0)
__global__ void z2_gather_split_kernel(const double* __restrict__ src, long long ld,
                                       const int* __restrict__ rowmap, int nrows,
                                       const int* __restrict__ colmap, int ncols,
                                       __nv_bfloat16* __restrict__ dst, long long piece_stride,
                                       int npieces) {
  long long total = (long long)nrows * ncols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / ncols), j = (int)(e - (long long)i * ncols);
    int cj = colmap[j];
    double x = cj >= 0 ? src[(long long)rowmap[i] * ld + cj] : 0.0;
    for (int p = 0; p < npieces; ++p) {
      __nv_bfloat16 b = __double2bfloat16(x);
      dst[p * piece_stride + e] = b;
      x -= (double)__bfloat162float(b);
    }
  }
}

// FP64 variant (the FP64 form): dst[i][j] = src[rowmap[i] * ld + colmap[j]]
__global__ void z2_gather_f64_kernel(const double* __restrict__ src, long long ld,
                                     const int* __restrict__ rowmap, int nrows,
                                     const int* __restrict__ colmap, int ncols,
                                     double* __restrict__ dst) {
  long long total = (long long)nrows * ncols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / ncols), j = (int)(e - (long long)i * ncols);
    int cj = colmap[j];
    dst[e] = cj >= 0 ? src[(long long)rowmap[i] * ld + cj] : 0.0;
  }
}

// BF16 pieces: dst[p][i][j] = src[p][rowmap[i]][colmap[j]] (0 where colmap[j] < 0)
__global__ void z2_gather_bf16_kernel(const __nv_bfloat16* __restrict__ src, long long ld,
                                      long long src_piece_stride, const int* __restrict__ rowmap,
                                      int nrows, const int* __restrict__ colmap, int ncols,
                                      __nv_bfloat16* __restrict__ dst, long long dst_piece_stride,
                                      int npieces) {
  long long total = (long long)nrows * ncols;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / ncols), j = (int)(e - (long long)i * ncols);
    int cj = colmap[j];
    long long so = (long long)rowmap[i] * ld + cj;
    for (int p = 0; p < npieces; ++p)
      dst[p * dst_piece_stride + e] = cj >= 0 ? src[p * src_piece_stride + so] : zero;
  }
}

// dense[r][n] = C_b[rowpos[r]][colpos[n]] if colpar[n] ^ q == rowpar[r] = b, else 0
template <typename T>
__global__ void z2_scatter_kernel(const T* __restrict__ c0, long long ld0, const T* __restrict__ c1,
                                  long long ld1, const int* __restrict__ rowblk,
                                  const int* __restrict__ rowpos, const int* __restrict__ colblk,
                                  const int* __restrict__ colpos, int q, int nrows, int ncols,
                                  T* __restrict__ dense) {
  long long total = (long long)nrows * ncols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / ncols), n = (int)(e - (long long)r * ncols);
    int b = rowblk[r];
    const T* cb = b == 0 ? c0 : c1;   // null: the block is empty (no columns)
    T v = T(0);
    if ((colblk[n] ^ q) == b && cb) v = cb[(long long)rowpos[r] * (b == 0 ? ld0 : ld1) + colpos[n]];
    dense[e] = v;
  }
}

// count[0] += number of elements of odd total parity that are not exactly zero.
// T is in slot layout: rows (slot 0 .. d-1), then columns (slot 0 .. d-1), slot 0
// slowest; bit v of mask[k] is the parity of index v of slot k.
__global__ void z2_check_kernel(const double* __restrict__ T, Z2Slots sl, unsigned long long total,
                                int* __restrict__ count) {
  int bad = 0;
  for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long r = e;
    unsigned p = 0;
    for (int k = 2 * sl.d - 1; k >= 0; --k) {
      const int s = k % sl.d;
      const unsigned sz = (unsigned)sl.chi[s];
      const unsigned idx = (unsigned)(r % sz);
      r /= sz;
      p ^= (sl.mask[s] >> idx) & 1u;
    }
    if (p && T[e] != 0.0) ++bad;
  }
  if (bad) atomicAdd(count, bad);
}

static unsigned grid_for(long long total) {
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}

void launch_z2_gather_split(const double* src, long long ld, const int* rowmap, int nrows,
                            const int* colmap, int ncols, __nv_bfloat16* dst, long long piece_stride,
                            int npieces, cudaStream_t s) {
  z2_gather_split_kernel<<<grid_for((long long)nrows * ncols), 256, 0, s>>>(
      src, ld, rowmap, nrows, colmap, ncols, dst, piece_stride, npieces);
  ++g_launches;
}

void launch_z2_gather_f64(const double* src, long long ld, const int* rowmap, int nrows,
                          const int* colmap, int ncols, double* dst, cudaStream_t s) {
  z2_gather_f64_kernel<<<grid_for((long long)nrows * ncols), 256, 0, s>>>(src, ld, rowmap, nrows,
                                                                           colmap, ncols, dst);
  ++g_launches;
}

void launch_z2_gather_bf16(const __nv_bfloat16* src, long long ld, long long src_piece_stride,
                           const int* rowmap, int nrows, const int* colmap, int ncols,
                           __nv_bfloat16* dst, long long dst_piece_stride, int npieces,
                           cudaStream_t s) {
  z2_gather_bf16_kernel<<<grid_for((long long)nrows * ncols), 256, 0, s>>>(
      src, ld, src_piece_stride, rowmap, nrows, colmap, ncols, dst, dst_piece_stride, npieces);
  ++g_launches;
}

void launch_z2_scatter_f32(const float* c0, long long ld0, const float* c1, long long ld1,
                           const int* rowblk, const int* rowpos, const int* colblk, const int* colpos,
                           int q, int nrows, int ncols, float* dense, cudaStream_t s) {
  z2_scatter_kernel<float><<<grid_for((long long)nrows * ncols), 256, 0, s>>>(
      c0, ld0, c1, ld1, rowblk, rowpos, colblk, colpos, q, nrows, ncols, dense);
  ++g_launches;
}

void launch_z2_scatter_f64(const double* c0, long long ld0, const double* c1, long long ld1,
                           const int* rowblk, const int* rowpos, const int* colblk, const int* colpos,
                           int q, int nrows, int ncols, double* dense, cudaStream_t s) {
  z2_scatter_kernel<double><<<grid_for((long long)nrows * ncols), 256, 0, s>>>(
      c0, ld0, c1, ld1, rowblk, rowpos, colblk, colpos, q, nrows, ncols, dense);
  ++g_launches;
}

void launch_z2_check(const double* T, const Z2Slots& sl, long long total, int* count, cudaStream_t s) {
  z2_check_kernel<<<grid_for(total), 256, 0, s>>>(T, sl, (unsigned long long)total, count);
  ++g_launches;
}

}  // namespace hotrg
