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
                                       void* __restrict__ dst, long long piece_stride,
                                       int npieces, int pfmt) {
  long long total = (long long)nrows * ncols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / ncols), j = (int)(e - (long long)i * ncols);
    int cj = colmap[j];
    double x = cj >= 0 ? src[(long long)rowmap[i] * ld + cj] : 0.0;
    store_pieces(dst, e, piece_stride, npieces, pfmt, x);
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

// Pieces (E = the bits of one BF16 or TF32 element): dst[p][i][j] = src[p][rowmap[i]][colmap[j]]
// (0 where colmap[j] < 0).  Rows over grid y, four consecutive columns per thread (ncols
// is a multiple of 4): one 4-element store per piece.
template <typename E, typename E4>
__global__ void z2_gather_pieces_kernel(const E* __restrict__ src, long long ld, long long src_piece_stride,
                                        const int* __restrict__ rowmap, int nrows,
                                        const int* __restrict__ colmap, int ncols, E* __restrict__ dst,
                                        long long dst_piece_stride, int npieces) {
  const int nq = ncols >> 2;
  for (int i = blockIdx.y; i < nrows; i += gridDim.y) {
    const E* sr = src + (long long)rowmap[i] * ld;
    E* dr = dst + (long long)i * ncols;
    for (int jq = blockIdx.x * blockDim.x + threadIdx.x; jq < nq; jq += gridDim.x * blockDim.x) {
      const int4 cm = reinterpret_cast<const int4*>(colmap)[jq];
      for (int p = 0; p < npieces; ++p) {
        const E* sp = sr + p * src_piece_stride;
        E4 v;
        v.x = cm.x >= 0 ? sp[cm.x] : E(0);
        v.y = cm.y >= 0 ? sp[cm.y] : E(0);
        v.z = cm.z >= 0 ? sp[cm.z] : E(0);
        v.w = cm.w >= 0 ? sp[cm.w] : E(0);
        *reinterpret_cast<E4*>(dr + p * dst_piece_stride + 4 * jq) = v;
      }
    }
  }
}

// dense[r][n] = C_b[rowpos[r]][colpos[n]] if colpar[n] ^ q == rowpar[r] = b, else 0.
// Rows over grid y, four consecutive columns per thread.
template <typename T>
__global__ void z2_scatter_kernel(const T* __restrict__ c0, long long ld0, const T* __restrict__ c1,
                                  long long ld1, const int* __restrict__ rowblk,
                                  const int* __restrict__ rowpos, const int* __restrict__ colblk,
                                  const int* __restrict__ colpos, int q, int nrows, int ncols,
                                  T* __restrict__ dense) {
  for (int r = blockIdx.y; r < nrows; r += gridDim.y) {
    const int b = rowblk[r];
    const T* cr = b == 0 ? c0 : c1;   // null: the block is empty (no columns)
    if (cr) cr += (long long)rowpos[r] * (b == 0 ? ld0 : ld1);
    T* dr = dense + (long long)r * ncols;
    for (int n0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x); n0 < ncols;
         n0 += 4 * gridDim.x * blockDim.x) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int n = n0 + u;
        if (n >= ncols) break;
        dr[n] = ((colblk[n] ^ q) == b && cr) ? cr[colpos[n]] : T(0);
      }
    }
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
                            const int* colmap, int ncols, void* dst, long long piece_stride,
                            int npieces, int pfmt, cudaStream_t s) {
  z2_gather_split_kernel<<<grid_for((long long)nrows * ncols), 256, 0, s>>>(
      src, ld, rowmap, nrows, colmap, ncols, dst, piece_stride, npieces, pfmt);
  ++g_launches;
}

void launch_z2_gather_f64(const double* src, long long ld, const int* rowmap, int nrows,
                          const int* colmap, int ncols, double* dst, cudaStream_t s) {
  z2_gather_f64_kernel<<<grid_for((long long)nrows * ncols), 256, 0, s>>>(src, ld, rowmap, nrows,
                                                                           colmap, ncols, dst);
  ++g_launches;
}

// rows over grid y (at most 65535, grid-stride beyond), columns over x
static dim3 grid_rows(int nrows, long long units_per_row) {
  long long bx = (units_per_row + 255) / 256;
  if (bx < 1) bx = 1;
  long long by = nrows < 1 ? 1 : nrows;
  if (by > 65535) by = 65535;
  // about 32 CTAs of 256 threads per SM in all
  long long cap = (152LL * 32 + by - 1) / by;
  if (bx > cap) bx = cap;
  return dim3((unsigned)bx, (unsigned)by);
}

void launch_z2_gather_pieces(const void* src, long long ld, long long src_piece_stride,
                             const int* rowmap, int nrows, const int* colmap, int ncols,
                             void* dst, long long dst_piece_stride, int npieces, int pfmt,
                             cudaStream_t s) {
  if (pfmt == PIECE_TF32)
    z2_gather_pieces_kernel<unsigned, uint4><<<grid_rows(nrows, ncols / 4), 256, 0, s>>>(
        (const unsigned*)src, ld, src_piece_stride, rowmap, nrows, colmap, ncols, (unsigned*)dst,
        dst_piece_stride, npieces);
  else
    z2_gather_pieces_kernel<unsigned short, ushort4><<<grid_rows(nrows, ncols / 4), 256, 0, s>>>(
        (const unsigned short*)src, ld, src_piece_stride, rowmap, nrows, colmap, ncols, (unsigned short*)dst,
        dst_piece_stride, npieces);
  ++g_launches;
}

void launch_z2_scatter_f32(const float* c0, long long ld0, const float* c1, long long ld1,
                           const int* rowblk, const int* rowpos, const int* colblk, const int* colpos,
                           int q, int nrows, int ncols, float* dense, cudaStream_t s) {
  z2_scatter_kernel<float><<<grid_rows(nrows, (ncols + 3) / 4), 256, 0, s>>>(
      c0, ld0, c1, ld1, rowblk, rowpos, colblk, colpos, q, nrows, ncols, dense);
  ++g_launches;
}

void launch_z2_scatter_f64(const double* c0, long long ld0, const double* c1, long long ld1,
                           const int* rowblk, const int* rowpos, const int* colblk, const int* colpos,
                           int q, int nrows, int ncols, double* dense, cudaStream_t s) {
  z2_scatter_kernel<double><<<grid_rows(nrows, (ncols + 3) / 4), 256, 0, s>>>(
      c0, ld0, c1, ld1, rowblk, rowpos, colblk, colpos, q, nrows, ncols, dense);
  ++g_launches;
}

void launch_z2_check(const double* T, const Z2Slots& sl, long long total, int* count, cudaStream_t s) {
  z2_check_kernel<<<grid_for(total), 256, 0, s>>>(T, sl, (unsigned long long)total, count);
  ++g_launches;
}

// Environment Grams in parity blocks (Sec. 3.2): X[i][k] = T[roff[i] + koff[k]], with the
// rows (n_j, current) and the summed index `rest` both listed even parity first, so that
// X[(rows of parity b)][(columns of parity b)] is a contiguous block and the Gram is
// block diagonal: S_b = X_b X_b^T.  One grid row per X row.
__global__ void z2_gather_rc_kernel(const double* __restrict__ T, const long long* __restrict__ roff,
                                    const long long* __restrict__ koff, long long K,
                                    double* __restrict__ X) {
  const long long ro = roff[blockIdx.y];
  double* xr = X + (long long)blockIdx.y * K;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < K;
       k += (long long)gridDim.x * blockDim.x)
    xr[k] = T[ro + koff[k]];
}

void launch_z2_gather_rc(const double* T, const long long* roff, int m, const long long* koff,
                         long long K, double* X, cudaStream_t s) {
  long long bx = (K + 255) / 256;
  const long long cap = (152LL * 16 + m - 1) / m;   // about 16 CTAs of 256 threads per SM
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  z2_gather_rc_kernel<<<dim3((unsigned)bx, (unsigned)m), 256, 0, s>>>(T, roff, koff, K, X);
  ++g_launches;
}

// S[i][j] = sum_z parts_b[z][min(p_i, p_j)][max(p_i, p_j)] if rows i and j are both of
// parity b (positions p_i, p_j in block b), else 0; parts_b holds ns_b split-K partials
// of the upper triangle of the m_b x m_b block Gram.
__global__ void z2_reduce_sym_kernel(const double* __restrict__ p0, int ns0, int m0,
                                     const double* __restrict__ p1, int ns1, int m1,
                                     const int* __restrict__ blk, const int* __restrict__ pos, int m,
                                     double* __restrict__ S) {
  const long long total = (long long)m * m;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e - (long long)i * m);
    double acc = 0.0;
    const int b = blk[i];
    if (b == blk[j]) {
      const int pi = pos[i], pj = pos[j];
      const int lo = pi < pj ? pi : pj, hi = pi < pj ? pj : pi;
      const double* p = b == 0 ? p0 : p1;
      const int mb = b == 0 ? m0 : m1, ns = b == 0 ? ns0 : ns1;
      const long long bb = (long long)mb * mb;
      for (int z = 0; z < ns; ++z) acc += p[z * bb + (long long)lo * mb + hi];
    }
    S[e] = acc;
  }
}

void launch_z2_reduce_sym(const double* p0, int ns0, int m0, const double* p1, int ns1, int m1,
                          const int* blk, const int* pos, int m, double* S, cudaStream_t s) {
  z2_reduce_sym_kernel<<<grid_for((long long)m * m), 256, 0, s>>>(p0, ns0, m0, p1, ns1, m1, blk, pos,
                                                                  m, S);
  ++g_launches;
}

// The derivative of a Gram from its parity blocks: dS[i][j] = sum_z (P_b[z][p_i][p_j] +
// P_b[z][p_j][p_i]) if rows i and j are both of parity b, else 0; P_b holds ns_b split-K
// partials of the full m_b x m_b block product dX_b X_b^T.
__global__ void z2_reduce_sum_t_kernel(const double* __restrict__ p0, int ns0, int m0,
                                       const double* __restrict__ p1, int ns1, int m1,
                                       const int* __restrict__ blk, const int* __restrict__ pos, int m,
                                       double* __restrict__ dS) {
  const long long total = (long long)m * m;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e - (long long)i * m);
    double acc = 0.0;
    const int b = blk[i];
    if (b == blk[j]) {
      const int pi = pos[i], pj = pos[j];
      const double* p = b == 0 ? p0 : p1;
      const int mb = b == 0 ? m0 : m1, ns = b == 0 ? ns0 : ns1;
      const long long bb = (long long)mb * mb;
      for (int z = 0; z < ns; ++z)
        acc += p[z * bb + (long long)pi * mb + pj] + p[z * bb + (long long)pj * mb + pi];
    }
    dS[e] = acc;
  }
}

void launch_z2_reduce_sum_t(const double* p0, int ns0, int m0, const double* p1, int ns1, int m1,
                            const int* blk, const int* pos, int m, double* dS, cudaStream_t s) {
  z2_reduce_sum_t_kernel<<<grid_for((long long)m * m), 256, 0, s>>>(p0, ns0, m0, p1, ns1, m1, blk, pos,
                                                                    m, dS);
  ++g_launches;
}

// Eigen-decomposition in parity blocks (Sec. 4.2.5): A^(j) is block diagonal in the
// parity of its composite index (hat, check), so each block is decomposed on its own.
// Ab[p][q] = A[rows[p]][rows[q]] for p, q < nb, zero-padded to npad x npad (a zero row and
// column of A adds an exact zero column to W = A V that no rotation ever touches)
__global__ void z2_gather_sym_kernel(const double* __restrict__ A, int n, const int* __restrict__ rows,
                                     int nb, int npad, double* __restrict__ Ab) {
  const int total = npad * npad;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int p = e / npad, q = e - p * npad;
    Ab[e] = (p < nb && q < nb) ? A[(long long)rows[p] * n + rows[q]] : 0.0;
  }
}

void launch_z2_gather_sym(const double* A, int n, const int* rows, int nb, int npad, double* Ab,
                          cudaStream_t s) {
  z2_gather_sym_kernel<<<grid_for((long long)npad * npad), 256, 0, s>>>(A, n, rows, nb, npad, Ab);
  ++g_launches;
}

// Column-major n x n M from the blocks (leading dimension ld): M[r + c n] =
// M_b[pos[r] + pos[c] ld] if rows r and c are both of parity b, else 0 (column c of M is
// column pos[c] of block blk[c]; the padding columns of the blocks are dropped)
__global__ void z2_scatter_eig_kernel(const double* __restrict__ m0, const double* __restrict__ m1,
                                      int ld, const int* __restrict__ blk, const int* __restrict__ pos,
                                      int n, double* __restrict__ M) {
  const int total = n * n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int cidx = e / n, r = e - cidx * n;
    const int b = blk[r];
    double v = 0.0;
    if (b == blk[cidx]) v = (b == 0 ? m0 : m1)[pos[r] + (long long)pos[cidx] * ld];
    M[e] = v;
  }
}

void launch_z2_scatter_eig(const double* m0, const double* m1, int ld, const int* blk, const int* pos,
                           int n, double* M, cudaStream_t s) {
  z2_scatter_eig_kernel<<<grid_for((long long)n * n), 256, 0, s>>>(m0, m1, ld, blk, pos, n, M);
  ++g_launches;
}

// dst[k] = max(src[a[k]], src[b[k]]) (b[k] < 0: src[a[k]] alone)
__global__ void z2_merge_sweeps_kernel(const int* __restrict__ src, SweepMerge m, int* __restrict__ dst) {
  const int k = threadIdx.x;
  if (k >= m.n) return;
  int v = m.a[k] >= 0 ? src[m.a[k]] : 0;
  if (m.b[k] >= 0 && src[m.b[k]] > v) v = src[m.b[k]];
  dst[k] = v;
}

void launch_z2_merge_sweeps(const int* src, const SweepMerge& m, int* dst, cudaStream_t s) {
  z2_merge_sweeps_kernel<<<1, 32, 0, s>>>(src, m, dst);
  ++g_launches;
}

}  // namespace hotrg
