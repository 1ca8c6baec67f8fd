// Internal declarations shared by the translation units of libhotrg.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>

namespace hotrg {

constexpr int kMaxD = 4;
constexpr int kMaxDevices = 64;  // per-device caches (SM counts, kernel attributes)
constexpr int kMaxDims = 10;     // tensor ranks handled by the index kernels
constexpr int kMaxBond = 64;

// Device-side state of a run; lives in device memory, read back on demand.
struct DevState {
  double kappa;        // K^(p) / 2^p
  double ln_tr;        // ln Tr T^(p) of the last new tensor (or of T^(0))
  double trace;        // Tr T^(p)
  double inv_trace;    // f^(p) = 1 / Tr T^(p)
  double ln_z_site;    // ln Z^(p) / 2^p
  double gu_wen;       // X of the last new tensor
  int status;          // 0 or a negative hotrg_status
  int p;               // steps taken (the step count of the last normalisation)
};

// Device-side derivative state of a run (d/d beta, forward mode), beside DevState.
struct TanState {
  double dkappa;       // d kappa_p / d beta
  double dln_tr;       // d ln Tr T^(p) / d beta
  double dln_z_site;   // d (ln Z^(p) / 2^p) / d beta
  double dtrace;       // Tr dT^(p)
  int degenerate;      // eigen pairs across the cut with no derivative (left out)
  int pad;
  double d2kappa;      // d^2 kappa_p / d beta^2 (second order carried)
  double d2ln_tr;      // d^2 ln Tr T^(p) / d beta^2
  double d2ln_z_site;  // d^2 (ln Z^(p) / 2^p) / d beta^2
};

// Per-leg results of the isometry selection.
struct LegResult {
  double eps[2];       // epsilon (A), epsilon' (A')
  double lam1[2];
  double gap;
  int chose_prime;
  int sweeps[2];
};

// Generic strided description of a tensor-times-isometry stage: every
// output element (over `ndim` free dims, plus the new index n) is
//   y = sum_{a in A(o), b} x[in(o) + a*ka_stride + b*kb_stride] * U[a + b*chi][n]
// with A(o) = {o[a_dim]} when a_dim >= 0 (the hat index stays free: prime
// side) and A(o) = [0, chi) when a_dim < 0 (both contracted: non-prime side).
struct ChainDesc {
  int ndim;
  int a_dim;
  int chi;             // chi_j (U has chi*chi rows)
  int nn;              // U columns used
  int ldu;             // row stride of U (>= nn)
  long long size[kMaxDims];
  long long in_stride[kMaxDims];
  long long out_stride[kMaxDims];
  long long ka_stride, kb_stride;
  long long n_out_stride;
  long long total;     // product of size[] (< 2^32)
  unsigned magic[kMaxDims];   // q = (umulhi(x, magic) + x) >> shift == x / size, 32-bit x
  int shift[kMaxDims];
  long long piece_stride;  // split outputs: distance between pieces (elements)
  int npieces;
  int pfmt;                // split outputs: PIECE_BF16 or PIECE_TF32
  int ctas_per_sm;         // grid cap of the launch: this many CTAs per SM (results do not depend on it)
};

// ---- operand pieces of the split forms: x = x_0 + x_1 + ..., x_0 = x rounded to the
// piece format, x_p = the remainder after x_0 .. x_{p-1}, rounded
enum { PIECE_BF16 = 0, PIECE_TF32 = 1 };
inline int piece_bytes(int pfmt) { return pfmt == PIECE_TF32 ? 4 : 2; }
// pieces per operand and their format for a split precision mode (enum hotrg_precision)
inline int split_pieces(int mode) { return mode == 1 || mode == 4 ? 2 : (mode == 3 ? 1 : 3); }
inline int split_format(int mode) { return mode >= 3 ? PIECE_TF32 : PIECE_BF16; }

// The piece products (terms) x_a y_b of the split GEMM: every term of order 2^-(8 or
// 11) x (a + b) up to the pieces' resolution (1 piece: 1 term; 2: 3; 3: 6).  Returns
// the number of terms.
inline int split_terms(int npieces, int* ta, int* tb) {
  static const int a1[1] = {0}, b1[1] = {0};
  static const int a2[3] = {1, 0, 0}, b2[3] = {0, 1, 0};
  static const int a3[6] = {2, 1, 0, 1, 0, 0}, b3[6] = {0, 1, 2, 0, 1, 0};
  const int n = npieces == 1 ? 1 : (npieces == 2 ? 3 : 6);
  const int* a = npieces == 1 ? a1 : (npieces == 2 ? a2 : a3);
  const int* b = npieces == 1 ? b1 : (npieces == 2 ? b2 : b3);
  for (int t = 0; t < n; ++t) {
    ta[t] = a[t];
    tb[t] = b[t];
  }
  return n;
}

#ifdef __CUDACC__
// x rounded to TF32 (10 stored mantissa bits, ties to even) in an FP32 word whose low
// 13 bits are zero; infinities and NaNs pass unchanged
__device__ __forceinline__ float round_tf32(float x) {
  unsigned u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;
  u += 0xfffu + ((u >> 13) & 1u);
  return __uint_as_float(u & 0xffffe000u);
}

__device__ __forceinline__ __nv_bfloat16 bf16_rn(float x) { return __float2bfloat16_rn(x); }
__device__ __forceinline__ __nv_bfloat16 bf16_rn(double x) { return __double2bfloat16(x); }

// x as npieces pieces of format PF: piece p at element off + p * pstride of o
template <int PF, typename T>
__device__ __forceinline__ void store_pieces_as(void* o, long long off, long long pstride, int npieces, T x) {
  if (PF == PIECE_TF32) {
    float* of = (float*)o + off;
    for (int p = 0; p < npieces; ++p) {
      const float v = round_tf32((float)x);
      of[p * pstride] = v;
      x -= (T)v;
    }
  } else {
    __nv_bfloat16* ob = (__nv_bfloat16*)o + off;
    for (int p = 0; p < npieces; ++p) {
      const __nv_bfloat16 v = bf16_rn(x);
      ob[p * pstride] = v;
      x -= (T)__bfloat162float(v);
    }
  }
}
template <typename T>
__device__ __forceinline__ void store_pieces(void* o, long long off, long long pstride, int npieces, int pfmt,
                                             T x) {
  if (pfmt == PIECE_TF32)
    store_pieces_as<PIECE_TF32>(o, off, pstride, npieces, x);
  else
    store_pieces_as<PIECE_BF16>(o, off, pstride, npieces, x);
}
#endif

// ---- kernels_tensor.cu
void launch_init_ising(double* T, int d, double beta, double h, cudaStream_t s);
void launch_permute(const double* in, double* out, int ndim, const long long* out_size,
                    const long long* in_stride, double scale, cudaStream_t s);
// FP64 (in, + in2 when given) -> npieces pieces of format pfmt
void launch_split(const double* in, long long rows, long long cols, long long ld_in, void* out,
                  long long ld_out, long long piece_stride, int npieces, int pfmt, cudaStream_t s,
                  const double* in2 = nullptr);
void launch_trace_y(const double* Tn, int chi_c, long long pn, double* Y, cudaStream_t s);
void launch_finish_step(double* Y, int chi_c, DevState* st, int p, int first, cudaStream_t s);
void launch_scale(const double* in, double* out, long long n, const DevState* st, cudaStream_t s);

// ---- kernels_env.cu
// FP64 FMA rate of the current device in TFLOP/s (CUDA events; 0 or a negative status)
int measure_fp64_rate(double* tflops);
// edge of the tiles of the symmetric (upper_only) FP64 products
int gram_tile();
// returns the number of split-K partials written
int launch_gemm_nt_f64(const double* A, long long lda, const double* B, long long ldb,
                       double* C, long long ldc, long long split_stride,
                       int M, int N, long long K, int nsplit, int upper_only, cudaStream_t s);
void launch_reduce_sym(const double* parts, int nsplit, int m, double* G, cudaStream_t s);
void launch_assemble_a(const double* s_hat, const double* s_chk, int chi_j, int chi_c,
                       double* A, cudaStream_t s);

// ---- kernels_eig.cu
// colmax: nmat (<= 16) words of scratch
int launch_jacobi(double* W, double* V, const double* A, int n, int nmat, int max_sweeps,
                  int* counters, unsigned long long* colmax, int* sweeps_out, DevState* st,
                  cudaStream_t s);
int launch_jacobi32_block(const double* A, float* W32, float* V32, int n, int nmat,
                          int max_sweeps, int* counters, cudaStream_t s);
void launch_widen_f32(const float* in, double* out, long long n, cudaStream_t s);
void launch_ns_coeff(double* G, int n, int nmat, cudaStream_t s);
void launch_gemm_nn_f64(const double* A, long long lda, const double* B, long long ldb, double* C,
                        long long ldc, int M, int N, int K, int batch, long long bsa,
                        long long bsb, long long bsc, cudaStream_t s);
void launch_gemm_nt_f64_batched(const double* A, long long lda, const double* B, long long ldb,
                                double* C, long long ldc, int M, int N, int K, int batch,
                                long long bsa, long long bsb, long long bsc, cudaStream_t s);
void launch_select(const double* W, const double* V, int n, int leg_index, int nnew,
                   double* lam_sorted, double* U64, float* U32, LegResult* res,
                   const int* sweeps, cudaStream_t s, int* rank_out = nullptr);

// ---- kernels_chain.cu
void launch_chain_f32(const ChainDesc& d, const void* in, int in_is_f64, const float* U,
                      void* out, int out_mode, cudaStream_t s);
void launch_chain_f64(const ChainDesc& d, const double* in, const double* U, double* out,
                      cudaStream_t s);
void launch_chain_f64acc(const ChainDesc& d, const void* in, int in_is_f64, const double* U,
                         void* out, int out_mode, cudaStream_t s);
// OUT_Z2_SPLIT_W: OUT_Z2_SPLIT for K lists whose length R is a multiple of 32 (every
// warp full, its threads in one row group of the output)
enum { OUT_F32 = 0, OUT_F64 = 1, OUT_BF16_SPLIT = 2, OUT_Z2_SPLIT = 3, OUT_Z2_SPLIT_W = 4 };

// Last prime stage written straight into the Z2 blocks of the bottleneck's B operand.
// The stage's out view is the dense B (row (n', n~) x kpad + k, k = (rho, n^')), whose
// leading free dims are exactly the k dims (R values).  Threads run over the K lists of
// both parities concatenated (kcat: dense k of list position x; block 0 = the first rb0
// positions), so the lanes of a warp hold consecutive positions of one block row.  An
// output goes to block b = parity(k) if its row's parity p_N satisfies p_N ^ q == b
// (the other half meets only zero blocks of T and is not formed), at row cpos[row] and
// column = the position of k in its list; split into pieces (format pfmt of the stage).
struct Z2Out {
  const int* kcat;        // dense k of every position of the two K lists (R entries)
  unsigned R;             // entries of kcat (product of the k dims)
  unsigned rb0;           // length of the parity-0 list
  const int* cblk;        // per column (n', n~) of this sub-slice: parity p_N
  const int* cpos;        // per column: position in the list of its parity
  int q;                  // parity of the c'-slice
  void* blk[2];           // the blocks
  long long ld[2];        // row pitch of block b (Kp_b)
  long long pstride[2];   // piece stride of block b
  long long kpad;         // row pitch of the dense out view
  long long nrow_step;    // rows between consecutive values of the stage's new index
  unsigned r_magic;       // t / R = (umulhi(t, r_magic) + t) >> r_shift
  int r_shift;
  long long rstride[kMaxDims];   // per free dim: its out stride / kpad (0 for the k dims)
};

// First non-prime stage read straight from the Z2 blocks of the bottleneck's product C.
// The stage's in strides are packed: (C row stride) << 32 | (C column stride).
struct Z2In {
  const int* rblk;   // per C row (c, n^): parity b
  const int* rpos;   // per C row: position in block b
  const int* cblk;   // per C column (n', n~) of this sub-slice: parity p_N
  const int* cpos;   // per C column: position in the list of its parity
  int q;             // parity of the c'-slice: row parity b pairs with p_N = b ^ q
  const float* c[2]; // the blocks (null if empty)
  long long ld;      // row pitch of the blocks
};
void launch_chain_f32_z2in(const ChainDesc& d, const Z2In& zi, const float* U, void* out, int out_mode,
                           cudaStream_t s);
void launch_chain_f32_z2out(const ChainDesc& d, const void* in, int in_is_f64, const float* U, const Z2Out& zo,
                            cudaStream_t s);

// ---- kernels_z2.cu
struct Z2Slots {
  int d;
  int chi[kMaxD];
  unsigned mask[kMaxD];   // bit v: parity of index v of the slot
};
void launch_z2_check(const double* T, const Z2Slots& sl, long long total, int* count, cudaStream_t s);
struct SweepMerge {
  int n;
  int a[2 * kMaxD], b[2 * kMaxD];
};
void launch_z2_gather_sym(const double* A, int n, const int* rows, int nb, int npad, double* Ab,
                          cudaStream_t s);
void launch_z2_scatter_eig(const double* m0, const double* m1, int ld, const int* blk, const int* pos,
                           int n, double* M, cudaStream_t s);
void launch_z2_merge_sweeps(const int* src, const SweepMerge& m, int* dst, cudaStream_t s);
void launch_z2_gather_rc(const double* T, const long long* roff, int m, const long long* koff,
                         long long K, double* X, cudaStream_t s);
void launch_z2_reduce_sym(const double* p0, int ns0, int m0, const double* p1, int ns1, int m1,
                          const int* blk, const int* pos, int m, double* S, cudaStream_t s);
void launch_z2_reduce_sum_t(const double* p0, int ns0, int m0, const double* p1, int ns1, int m1,
                            const int* blk, const int* pos, int m, double* dS, cudaStream_t s);
void launch_z2_gather_split(const double* src, long long ld, const int* rowmap, int nrows,
                            const int* colmap, int ncols, void* dst, long long piece_stride,
                            int npieces, int pfmt, cudaStream_t s);
void launch_z2_gather_f64(const double* src, long long ld, const int* rowmap, int nrows,
                          const int* colmap, int ncols, double* dst, cudaStream_t s);
// gathers pieces of either format (a copy of their bits)
void launch_z2_gather_pieces(const void* src, long long ld, long long src_piece_stride,
                             const int* rowmap, int nrows, const int* colmap, int ncols,
                             void* dst, long long dst_piece_stride, int npieces, int pfmt,
                             cudaStream_t s);
void launch_z2_scatter_f32(const float* c0, long long ld0, const float* c1, long long ld1,
                           const int* rowblk, const int* rowpos, const int* colblk, const int* colpos,
                           int q, int nrows, int ncols, float* dense, cudaStream_t s);
void launch_z2_scatter_f64(const double* c0, long long ld0, const double* c1, long long ld1,
                           const int* rowblk, const int* rowpos, const int* colblk, const int* colpos,
                           int q, int nrows, int ncols, double* dense, cudaStream_t s);

// ---- kernels_tc_gemm.cu
// C[M][N] (fp32, ldc) = sum_t Apiece[pa_t] (M x Kpad) . Bpiece[pb_t] (N x Kpad)^T,
// pieces of format pfmt; Kpad a multiple of 32 (BF16) or of 32 (TF32, pair form only)
int launch_tc_gemm(const void* A, int M, const void* B, int N, int Kpad, int npieces, int nterms,
                   const int* pa, const int* pb, float* C, long long ldc, int* err_flag, cudaStream_t s,
                   float* ms_out, int pfmt = PIECE_BF16);
int tc_gemm_ready();
// milliseconds per launch of the split GEMM on device-resident operands (rate probe)
int measure_tc_gemm_rate(int npieces, int M, int N, int Kpad, int iters, double* ms_per_launch,
                         int pfmt = PIECE_BF16);

// ---- kernels_tensor.cu: streaming multiprocessors of the current device (cached per device)
int sm_count();

extern std::atomic<long long> g_launches;   // kernels launched by this library
// ---- kernels_tangent.cu (d/d beta in forward mode)
void launch_init_ising_dbeta(double* dT, int d, double beta, double h, cudaStream_t s);
void launch_sym_sum(const double* parts, int nsplit, int m, double* dS, cudaStream_t s);
void launch_assemble_dot(const double* sh, const double* dsh, const double* sc, const double* dsc, int chi_j,
                         int chi_c, double* dA, cudaStream_t s);
void launch_eig_dscale(const double* Z, const double* lam_sorted, const int* rank, int n, int nnew,
                       double rel_tol, double* Zt, TanState* tst, cudaStream_t s);
void launch_transpose(const double* in, int rows, int cols, double* out, cudaStream_t s);
void launch_axpby(double a, const double* x, double b, double* y, long long n, cudaStream_t s);
void launch_add_f32(const float* x, float* y, long long n, cudaStream_t s);
void launch_narrow_f64(const double* in, float* out, long long n, cudaStream_t s);
void launch_finish_tangent(const double* Yd, int chi_c, const DevState* st, TanState* tst, int p, int first,
                           cudaStream_t s);
void launch_tangent_scale(const double* dT, const double* That, double* out, long long n, const DevState* st,
                          const TanState* tst, cudaStream_t s);
// second order (d^2 / d beta^2)
void launch_init_ising_d2beta(double* d2T, int d, double beta, double h, cudaStream_t s);
void launch_assemble_ddot(const double* sh, const double* dsh, const double* d2sh, const double* sc,
                          const double* dsc, const double* d2sc, int chi_j, int chi_c, double* d2A, cudaStream_t s);
void launch_eig_d2(const double* G1, const double* Gs, const double* G2s, const double* lam_sorted, const int* rank,
                   int n, int nnew, double rel_tol, double* Z2t, cudaStream_t s);
void launch_finish_tangent2(const double* Yd2, int chi_c, const DevState* st, TanState* tst, int p, int first,
                            cudaStream_t s);
void launch_tangent2_scale(const double* d2T, const double* dT, const double* dThat, const double* That, double* out,
                           long long n, const DevState* st, const TanState* tst, cudaStream_t s);

}  // namespace hotrg
