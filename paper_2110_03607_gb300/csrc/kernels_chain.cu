// Tensor-times-isometry stages of the new-tensor contraction (Sec. 4.2.9):
//  * prime side, Eqs. (TU1)-(TUNCD): sum over n-check'_j of
//    U~^(j)_{(n^'_j n~'_j), n'_j} C~ -- the hat index n^'_j stays free;
//  * non-prime side, Eqs. (AfterBNNCD)-(AfterBN1): sum over (n^_j, n~_j) of
//    U~^(j)_{(n^_j n~_j), n_j} C^.
// A stage is described by a ChainDesc (strides of every free index in the
// input and output, strides of the contracted hat/check indices).  Each
// thread owns one free multi-index and accumulates all chi_j^new outputs in
// registers; U~^(j) sits in shared memory (padded rows, see URow).
#include "hotrg_internal.cuh"

namespace hotrg {

// Row pitch of U~ in shared memory.  FP32: NN + 4 words keeps every row 16-byte
// aligned for float4 loads (one LDS.128 per four FMAs) and puts the rows of eight
// consecutive hat indices (lanes of the prime side) on distinct bank groups.  FP64:
// NN + 1 words, scalar loads.
template <typename TAcc, int NN>
struct URow {
  static constexpr int ld = NN + 1;
  __device__ __forceinline__ static void fma_row(TAcc x, const TAcc* ur, TAcc* acc) {
#pragma unroll
    for (int n = 0; n < NN; ++n) acc[n] = fma(x, ur[n], acc[n]);
  }
};
template <int NN>
struct URow<float, NN> {
  static constexpr int ld = NN + 4;
  __device__ __forceinline__ static void fma_row(float x, const float* ur, float* acc) {
#pragma unroll
    for (int n = 0; n < NN; n += 4) {
      const float4 u = *reinterpret_cast<const float4*>(ur + n);
      acc[n] = fmaf(x, u.x, acc[n]);
      acc[n + 1] = fmaf(x, u.y, acc[n + 1]);
      acc[n + 2] = fmaf(x, u.z, acc[n + 2]);
      acc[n + 3] = fmaf(x, u.w, acc[n + 3]);
    }
  }
};

// The stages that read the Z2 blocks of C and write those of B are held to three and
// four CTAs per SM (80 and 64 registers): both are bound by memory latency.  Wider
// accumulator rows (24, 32 outputs) or FP64 inputs take three or two, without spills.
template <typename TIn, int NN, int OUT, bool ZIN>
constexpr int chain_min_ctas() {
  return ZIN ? (NN <= 16 ? 3 : 2)
             : (OUT == OUT_Z2_SPLIT || OUT == OUT_Z2_SPLIT_W)
                   ? (NN <= 16 ? (sizeof(TIn) == 4 ? 4 : 3) : (NN <= 24 && sizeof(TIn) == 4 ? 3 : 2))
                   : 1;
}

// ZW (with ZIN): the 32 threads of a warp read the same rows of C (the host checks the
// thread dims: the leading dims without a row stride span a multiple of 32 threads, and
// so does the total); lane a then reads row a's block and position once, before the sums
template <typename TIn, typename TAcc, int NN, int OUT, bool ZIN = false, bool ZW = false>
__global__ void __launch_bounds__(256, (chain_min_ctas<TIn, NN, OUT, ZIN>())) chain_kernel(ChainDesc d, const TIn* __restrict__ in,
                                                    const TAcc* __restrict__ U, void* out, Z2In zi,
                                                    Z2Out zo) {
  extern __shared__ __align__(16) unsigned char smem_u[];
  TAcc* us = reinterpret_cast<TAcc*>(smem_u);
  const int rows = d.chi * d.chi;
  constexpr int ld = URow<TAcc, NN>::ld;
  for (int e = threadIdx.x; e < rows * NN; e += blockDim.x) {
    int r = e / NN, c = e % NN;
    us[r * ld + c] = c < d.nn ? U[r * d.ldu + c] : TAcc(0);
  }
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < d.total; t += stride) {
    unsigned rem = (unsigned)t;
    unsigned kidx = 0;
    if (OUT == OUT_Z2_SPLIT || OUT == OUT_Z2_SPLIT_W) {
      // t = (row group, list position): the thread's dense k comes from the K lists
      const unsigned grp = (unsigned)(((unsigned long long)__umulhi(rem, zo.r_magic) + rem) >> zo.r_shift);
      kidx = rem - grp * zo.R;
      rem = grp * zo.R + (unsigned)zo.kcat[kidx];
    }
    long long in_off = 0, out_off = 0, orow = 0;   // orow: the output row (Z2 outputs)
    int a_val = 0;
#pragma unroll
    for (int k = 0; k < kMaxDims; ++k) {
      if (k >= d.ndim) break;
      // rem / size[k] by multiply-shift (sizes and magics prepared on the host)
      unsigned q = (unsigned)(((unsigned long long)__umulhi(rem, d.magic[k]) + rem) >> d.shift[k]);
      unsigned idx = rem - q * (unsigned)d.size[k];
      rem = q;
      in_off += (long long)idx * d.in_stride[k];
      out_off += (long long)idx * d.out_stride[k];
      if (OUT == OUT_Z2_SPLIT || OUT == OUT_Z2_SPLIT_W) orow += (long long)idx * zo.rstride[k];
      if (k == d.a_dim) a_val = (int)idx;
    }
    // OUT_Z2_SPLIT_W: the warp's threads share the output rows row0 + n nrow_step; lane n
    // reads the packed (position | block << 31) of row n now, so that the lookups'
    // latency hides behind the multiply-adds, and the stores take them by shuffle
    unsigned zlane = 0u;
    if (OUT == OUT_Z2_SPLIT_W) {
      const int ln = threadIdx.x & 31;
      if (ln < NN && ln < d.nn) {
        const long long row = orow + ln * zo.nrow_step;
        zlane = (unsigned)zo.cpos[row] | ((unsigned)(zo.cblk[row] ^ zo.q) << 31);
      }
    }
    TAcc acc[NN];
#pragma unroll
    for (int n = 0; n < NN; ++n) acc[n] = TAcc(0);
    const int a_lo = d.a_dim >= 0 ? a_val : 0;
    const int a_hi = d.a_dim >= 0 ? a_val + 1 : d.chi;
    if (d.a_dim >= 0) {
      // prime side: one hat index, chi terms
      const TIn* xa = in + in_off;
      for (int b = 0; b < d.chi; ++b) {
        TAcc x = (TAcc)xa[(long long)b * d.kb_stride];
        const TAcc* ur = us + (a_val + b * d.chi) * ld;
        URow<TAcc, NN>::fma_row(x, ur, acc);
      }
    } else if (ZIN) {
      // non-prime side from the Z2 blocks of C: only columns of parity (row parity) ^ q
      // are nonzero; same two-level sums
      const long long row0 = in_off >> 32, kar = d.ka_stride >> 32;
      const long long col0 = in_off & 0xffffffffLL;
      unsigned zr = 0u;
      if (ZW) {
        const int ln = threadIdx.x & 31;
        if (ln < d.chi) {
          const long long row = row0 + ln * kar;
          zr = (unsigned)zi.rpos[row] | ((unsigned)zi.rblk[row] << 31);
        }
      }
      // the column maps do not depend on a: for chi <= 16 read them once, packed as
      // position | (block of the column) << 31
      unsigned cpk[16];
      const bool hoist = d.chi <= 16;
      if (hoist) {
#pragma unroll
        for (int b = 0; b < 16; ++b) {
          if (b < d.chi) {
            const long long col = col0 + b * d.kb_stride;
            cpk[b] = (unsigned)zi.cpos[col] | ((unsigned)(zi.cblk[col] ^ zi.q) << 31);
          } else {
            cpk[b] = 0u;
          }
        }
      }
      for (int a = a_lo; a < a_hi; ++a) {
        int rb;
        long long rp;
        if (ZW) {   // warp-uniform: the continue below is taken by the whole warp
          const unsigned z = __shfl_sync(0xffffffffu, zr, a);
          rb = (int)(z >> 31);
          rp = (long long)(z & 0x7fffffffu);
        } else {
          const long long row = row0 + a * kar;
          rb = zi.rblk[row];
          rp = zi.rpos[row];
        }
        const float* cr = rb ? zi.c[1] : zi.c[0];
        if (!cr) continue;
        cr += rp * zi.ld;
        TAcc part[NN];
#pragma unroll
        for (int n = 0; n < NN; ++n) part[n] = TAcc(0);
        if (hoist) {
#pragma unroll
          for (int b = 0; b < 16; ++b) {
            if (b >= d.chi) break;
            if ((int)(cpk[b] >> 31) != rb) continue;
            TAcc x = (TAcc)cr[cpk[b] & 0x7fffffffu];
            URow<TAcc, NN>::fma_row(x, us + (a + b * d.chi) * ld, part);
          }
        } else {
          for (int b = 0; b < d.chi; ++b) {
            const long long col = col0 + b * d.kb_stride;
            if ((zi.cblk[col] ^ zi.q) != rb) continue;
            TAcc x = (TAcc)cr[zi.cpos[col]];
            const TAcc* ur = us + (a + b * d.chi) * ld;
            URow<TAcc, NN>::fma_row(x, ur, part);
          }
        }
#pragma unroll
        for (int n = 0; n < NN; ++n) acc[n] += part[n];
      }
    } else
    // non-prime side, chi^2 terms, summed in two levels: the chi terms over b go
    // into a fresh partial that is then added once (rounding ~2 sqrt(chi), not chi)
    for (int a = a_lo; a < a_hi; ++a) {
      const TIn* xa = in + in_off + (long long)a * d.ka_stride;
      TAcc part[NN];
#pragma unroll
      for (int n = 0; n < NN; ++n) part[n] = TAcc(0);
      for (int b = 0; b < d.chi; ++b) {
        TAcc x = (TAcc)xa[(long long)b * d.kb_stride];
        const TAcc* ur = us + (a + b * d.chi) * ld;
        URow<TAcc, NN>::fma_row(x, ur, part);
      }
#pragma unroll
      for (int n = 0; n < NN; ++n) acc[n] += part[n];
    }
    if (OUT == OUT_F32) {
      float* o = (float*)out;
#pragma unroll
      for (int n = 0; n < NN; ++n)
        if (n < d.nn) o[out_off + n * d.n_out_stride] = (float)acc[n];
    } else if (OUT == OUT_F64) {
      double* o = (double*)out;
#pragma unroll
      for (int n = 0; n < NN; ++n)
        if (n < d.nn) o[out_off + n * d.n_out_stride] = (double)acc[n];
    } else if (OUT == OUT_BF16_SPLIT) {
      // the format branch outside the unrolled loop keeps one copy of it live
      if (d.pfmt == PIECE_TF32) {
#pragma unroll
        for (int n = 0; n < NN; ++n) {
          if (n >= d.nn) break;
          store_pieces_as<PIECE_TF32>(out, out_off + n * d.n_out_stride, d.piece_stride, d.npieces, acc[n]);
        }
      } else {
#pragma unroll
        for (int n = 0; n < NN; ++n) {
          if (n >= d.nn) break;
          store_pieces_as<PIECE_BF16>(out, out_off + n * d.n_out_stride, d.piece_stride, d.npieces, acc[n]);
        }
      }
    } else {
      // OUT_Z2_SPLIT: consecutive threads hold consecutive positions of one K list, so
      // a warp's stores to a block row are contiguous
      const long long row0 = orow;
      const int kb = kidx >= zo.rb0 ? 1 : 0;
      const long long kpos = (long long)(kb ? kidx - zo.rb0 : kidx);
      // selects, not an index: an indexed parameter array would be copied to local memory
      void* ob = kb ? zo.blk[1] : zo.blk[0];
      const long long ld = kb ? zo.ld[1] : zo.ld[0], ps = kb ? zo.pstride[1] : zo.pstride[0];
      if (OUT == OUT_Z2_SPLIT_W) {
        if (d.pfmt == PIECE_TF32) {
#pragma unroll
          for (int n = 0; n < NN; ++n) {
            if (n >= d.nn) break;
            const unsigned z = __shfl_sync(0xffffffffu, zlane, n);
            if ((int)(z >> 31) != kb) continue;
            store_pieces_as<PIECE_TF32>(ob, kpos + (long long)(z & 0x7fffffffu) * ld, ps, d.npieces, acc[n]);
          }
        } else {
#pragma unroll
          for (int n = 0; n < NN; ++n) {
            if (n >= d.nn) break;
            const unsigned z = __shfl_sync(0xffffffffu, zlane, n);
            if ((int)(z >> 31) != kb) continue;
            store_pieces_as<PIECE_BF16>(ob, kpos + (long long)(z & 0x7fffffffu) * ld, ps, d.npieces, acc[n]);
          }
        }
      } else if (d.pfmt == PIECE_TF32) {
#pragma unroll
        for (int n = 0; n < NN; ++n) {
          if (n >= d.nn) break;
          const long long row = row0 + n * zo.nrow_step;
          if ((zo.cblk[row] ^ zo.q) != kb) continue;
          store_pieces_as<PIECE_TF32>(ob, kpos + (long long)zo.cpos[row] * ld, ps, d.npieces, acc[n]);
        }
      } else {
#pragma unroll
        for (int n = 0; n < NN; ++n) {
          if (n >= d.nn) break;
          const long long row = row0 + n * zo.nrow_step;
          if ((zo.cblk[row] ^ zo.q) != kb) continue;
          store_pieces_as<PIECE_BF16>(ob, kpos + (long long)zo.cpos[row] * ld, ps, d.npieces, acc[n]);
        }
      }
    }
  }
}

template <typename TIn, typename TAcc, int NN, int OUT, bool ZIN = false, bool ZW = false>
static void launch_one(const ChainDesc& d, const TIn* in, const TAcc* U, void* out, cudaStream_t s,
                       const Z2In& zi = Z2In{}, const Z2Out& zo = Z2Out{}) {
  size_t smem = (size_t)d.chi * d.chi * URow<TAcc, NN>::ld * sizeof(TAcc);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(chain_kernel<TIn, TAcc, NN, OUT, ZIN, ZW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  long long blocks = (d.total + 255) / 256;
  const long long cap = (long long)(d.ctas_per_sm > 0 ? d.ctas_per_sm : 16) * sm_count();
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  chain_kernel<TIn, TAcc, NN, OUT, ZIN, ZW><<<(unsigned)blocks, 256, smem, s>>>(d, in, U, out, zi, zo);
  ++g_launches;
}

template <typename TIn, typename TAcc, int NN>
static void dispatch_out(const ChainDesc& d, const TIn* in, const TAcc* U, void* out, int out_mode,
                         cudaStream_t s) {
  if (out_mode == OUT_F32) launch_one<TIn, TAcc, NN, OUT_F32>(d, in, U, out, s);
  else if (out_mode == OUT_F64) launch_one<TIn, TAcc, NN, OUT_F64>(d, in, U, out, s);
  else launch_one<TIn, TAcc, NN, OUT_BF16_SPLIT>(d, in, U, out, s);
}

template <typename TIn, typename TAcc>
static void dispatch_nn(const ChainDesc& d, const TIn* in, const TAcc* U, void* out, int out_mode,
                        cudaStream_t s) {
  if (d.nn <= 4) dispatch_out<TIn, TAcc, 4>(d, in, U, out, out_mode, s);
  else if (d.nn <= 8) dispatch_out<TIn, TAcc, 8>(d, in, U, out, out_mode, s);
  else if (d.nn <= 16) dispatch_out<TIn, TAcc, 16>(d, in, U, out, out_mode, s);
  else if (d.nn <= 24) dispatch_out<TIn, TAcc, 24>(d, in, U, out, out_mode, s);
  else dispatch_out<TIn, TAcc, 32>(d, in, U, out, out_mode, s);
}

template <int OUT, bool ZW>
static void dispatch_nn_z2in(const ChainDesc& d, const Z2In& zi, const float* U, void* out, cudaStream_t s) {
  const float* none = nullptr;
  if (d.nn <= 4) launch_one<float, float, 4, OUT, true, ZW>(d, none, U, out, s, zi);
  else if (d.nn <= 8) launch_one<float, float, 8, OUT, true, ZW>(d, none, U, out, s, zi);
  else if (d.nn <= 16) launch_one<float, float, 16, OUT, true, ZW>(d, none, U, out, s, zi);
  else if (d.nn <= 24) launch_one<float, float, 24, OUT, true, ZW>(d, none, U, out, s, zi);
  else launch_one<float, float, 32, OUT, true, ZW>(d, none, U, out, s, zi);
}

void launch_chain_f32_z2in(const ChainDesc& d, const Z2In& zi, const float* U, void* out, int out_mode,
                           cudaStream_t s) {
  // warp-uniform rows of C: thread t's leading indices (those without a row stride)
  // span p0 threads; with p0 and the total multiples of 32 every warp is full and its
  // threads differ only in those indices
  long long p0 = 1;
  for (int k = 0; k < d.ndim && (d.in_stride[k] >> 32) == 0; ++k) p0 *= d.size[k];
  const bool zw = p0 % 32 == 0 && d.total % 32 == 0 && d.chi <= 32;
  if (out_mode == OUT_F64) {
    if (zw) dispatch_nn_z2in<OUT_F64, true>(d, zi, U, out, s);
    else dispatch_nn_z2in<OUT_F64, false>(d, zi, U, out, s);
  } else {
    if (zw) dispatch_nn_z2in<OUT_F32, true>(d, zi, U, out, s);
    else dispatch_nn_z2in<OUT_F32, false>(d, zi, U, out, s);
  }
}

template <typename TIn, int OUT>
static void dispatch_nn_z2out(const ChainDesc& d, const TIn* in, const float* U, const Z2Out& zo, cudaStream_t s) {
  const Z2In none{};
  if (d.nn <= 4) launch_one<TIn, float, 4, OUT>(d, in, U, nullptr, s, none, zo);
  else if (d.nn <= 8) launch_one<TIn, float, 8, OUT>(d, in, U, nullptr, s, none, zo);
  else if (d.nn <= 16) launch_one<TIn, float, 16, OUT>(d, in, U, nullptr, s, none, zo);
  else if (d.nn <= 24) launch_one<TIn, float, 24, OUT>(d, in, U, nullptr, s, none, zo);
  else launch_one<TIn, float, 32, OUT>(d, in, U, nullptr, s, none, zo);
}

void launch_chain_f32_z2out(const ChainDesc& d, const void* in, int in_is_f64, const float* U, const Z2Out& zo,
                            cudaStream_t s) {
  // R a multiple of 32: thread t of the grid covers list position t % R of row group
  // t / R, so the 32 threads of a warp share the row group, and d.total (row groups x R)
  // leaves no warp partly filled
  const bool warp_rows = zo.R % 32u == 0;
  if (in_is_f64) {
    if (warp_rows) dispatch_nn_z2out<double, OUT_Z2_SPLIT_W>(d, (const double*)in, U, zo, s);
    else dispatch_nn_z2out<double, OUT_Z2_SPLIT>(d, (const double*)in, U, zo, s);
  } else {
    if (warp_rows) dispatch_nn_z2out<float, OUT_Z2_SPLIT_W>(d, (const float*)in, U, zo, s);
    else dispatch_nn_z2out<float, OUT_Z2_SPLIT>(d, (const float*)in, U, zo, s);
  }
}

void launch_chain_f32(const ChainDesc& d, const void* in, int in_is_f64, const float* U, void* out,
                      int out_mode, cudaStream_t s) {
  if (in_is_f64) dispatch_nn<double, float>(d, (const double*)in, U, out, out_mode, s);
  else dispatch_nn<float, float>(d, (const float*)in, U, out, out_mode, s);
}

// FP64 accumulation: the FP64 form of the step (double in, double out), and the
// FP64-chain variant of the split form (double or float in, any output).
void launch_chain_f64acc(const ChainDesc& d, const void* in, int in_is_f64, const double* U, void* out,
                         int out_mode, cudaStream_t s) {
  if (in_is_f64) dispatch_nn<double, double>(d, (const double*)in, U, out, out_mode, s);
  else dispatch_nn<float, double>(d, (const float*)in, U, out, out_mode, s);
}

void launch_chain_f64(const ChainDesc& d, const double* in, const double* U, double* out,
                      cudaStream_t s) {
  dispatch_nn<double, double>(d, in, U, out, OUT_F64, s);
}

}  // namespace hotrg
