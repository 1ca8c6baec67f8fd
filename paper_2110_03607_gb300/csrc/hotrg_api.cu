// C ABI of libhotrg: context, device memory, and the orchestration of one
// HOTRG coarse-graining step on one stream (Sec. 4.2 of Yamashita & Sakurai,
// arXiv:2110.03607).
//
// Device layout of the local tensor ("slot layout"): a row-major matrix
// T[(i_0, .., i_{d-1})][(i_0', .., i_{d-1}')] whose slot s holds lattice axis
// order[s].  A step along `axis` first permutes T so that slot 0 is the
// Current direction (c, c') and slot j is Next j (n_j, n_j') -- the index
// naming of Secs. 3.1.2-3.1.3.  In that layout T is at the same time the
// c-fixed tensors (rows c) and the c'-fixed tensors (column blocks c') of
// Sec. 3.2, so the bottleneck of Eq. (BottleneckPart) is one GEMM with T as
// its left operand, sliced over c'.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <system_error>
#include <thread>
#include <map>
#include <vector>

#include "hotrg_internal.cuh"
#include "../../include/hotrg.h"

using namespace hotrg;

namespace {

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

// index names for the chain descriptors
enum : int {
  I_C = 1,
  I_RHO = 2,
  I_NH = 10,   // n^_j   (hat copy, unprimed)
  I_NC = 20,   // n~_j   (check copy, unprimed)
  I_NHP = 30,  // n^'_j  (hat copy, primed)
  I_NCP = 40,  // n~'_j  (check copy, primed)
  I_N = 50,    // n_j    (new, unprimed)
  I_NP = 60    // n'_j   (new, primed)
};

struct Ix {
  int name;
  long long size;
  long long stride;
};
typedef std::vector<Ix> View;

View contiguous(const std::vector<std::pair<int, long long>>& names) {
  View v(names.size());
  long long st = 1;
  for (int k = (int)names.size() - 1; k >= 0; --k) {
    v[k] = {names[k].first, names[k].second, st};
    st *= names[k].second;
  }
  return v;
}

long long stride_of(const View& v, int name, bool* found = nullptr) {
  for (auto& x : v)
    if (x.name == name) {
      if (found) *found = true;
      return x.stride;
    }
  if (found) *found = false;
  return 0;
}

// Returns false if the free dimensions do not fit the descriptor.
bool make_stage(ChainDesc& d, const View& in, const View& out, int a_name, int b_name, int n_name,
                int chi, int nn) {
  memset(&d, 0, sizeof(d));
  struct Fd {
    int name;
    long long size, ist, ost;
  };
  std::vector<Fd> fr;
  for (auto& o : out)
    if (o.name != n_name && o.size > 1) fr.push_back({o.name, o.size, stride_of(in, o.name), o.stride});
  for (auto& o : out)
    if (o.name == a_name && o.size == 1) fr.push_back({o.name, 1, 0, o.stride});
  std::stable_sort(fr.begin(), fr.end(), [](const Fd& a, const Fd& b) { return a.ost < b.ost; });
  // merge neighbours that are contiguous in both input and output (never the hat index)
  std::vector<Fd> mg;
  for (auto& f : fr) {
    if (!mg.empty()) {
      Fd& b = mg.back();
      if (b.name != a_name && f.name != a_name && f.ost == b.ost * b.size && f.ist == b.ist * b.size) {
        b.size *= f.size;
        continue;
      }
    }
    mg.push_back(f);
  }
  if ((int)mg.size() > kMaxDims) return false;
  d.ndim = (int)mg.size();
  d.a_dim = -1;
  d.total = 1;
  for (int k = 0; k < d.ndim; ++k) {
    d.size[k] = mg[k].size;
    d.out_stride[k] = mg[k].ost;
    d.in_stride[k] = mg[k].ist;
    if (mg[k].name == a_name) d.a_dim = k;
    d.total *= mg[k].size;
  }
  d.ka_stride = d.a_dim >= 0 ? 0 : stride_of(in, a_name);
  d.kb_stride = stride_of(in, b_name);
  d.n_out_stride = stride_of(out, n_name);
  d.chi = chi;
  d.nn = nn;
  d.ldu = nn;
  d.npieces = 1;
  d.pfmt = PIECE_BF16;
  d.ctas_per_sm = 16;
  if (d.total >= (1LL << 32)) return false;
  for (int k = 0; k < d.ndim; ++k) {
    // Hacker's Delight unsigned division by an invariant: l = ceil(log2 s),
    // m = floor(2^32 (2^l - s) / s) + 1, x / s = (umulhi(x, m) + x) >> l
    unsigned long long sz = (unsigned long long)d.size[k];
    int l = 0;
    while ((1ULL << l) < sz) ++l;
    d.shift[k] = l;
    d.magic[k] = (unsigned)((((1ULL << l) - sz) << 32) / sz + 1);
  }
  return true;
}

}  // namespace

struct hotrg_ctx {
  int d = 0;
  double beta = 0.0;
  int chis[kMaxD] = {0, 0, 0, 0};
  int order[kMaxD] = {0, 1, 2, 3};
  int p = 0;
  int precision = HOTRG_PREC_BF16X6;
  cudaStream_t stream = nullptr;
  hotrg_alloc_fn afn = nullptr;
  hotrg_free_fn ffn = nullptr;
  void* user = nullptr;
  int poisoned = 0;
  size_t held = 0;
  double fp64_below = 68719476736.0;  // 2^36 flops
  double slice_budget_bytes = 160e9;   // cap on the per-(sub)slice operands
  // diagnostic: FP64-accumulating chains around the split-BF16 bottleneck
  int f64_chains = getenv("HOTRG_DEBUG_F64_CHAINS") ? atoi(getenv("HOTRG_DEBUG_F64_CHAINS")) : 0;
  // phase timing
  int profile = 0;
  int last_fp64 = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
  std::vector<cudaEvent_t> event_pool;
  size_t event_next = 0;
  // last step
  int last_valid = 0;
  int last_nlegs = 0;
  int last_leg_axis[kMaxD - 1] = {0, 0, 0};
  int last_leg_n[kMaxD - 1] = {0, 0, 0};
  int last_leg_nnew[kMaxD - 1] = {0, 0, 0};
  long long last_lam_off[kMaxD - 1] = {0, 0, 0};
  long long last_u_off[kMaxD - 1] = {0, 0, 0};
  // Z2 block structure: the parity of every index of every axis (both legs of an
  // axis share it), known while z2_valid; used for the contraction while z2_enabled
  int z2_enabled = 1;
  int z2_valid = 0;
  std::vector<unsigned char> par[kMaxD];
  int last_z2 = 0;
  double last_bn_dense = 0.0, last_bn_done = 0.0;
  // pinned host staging for index maps, reused once the copy recorded in hpin_ev is done
  void* hpin = nullptr;
  size_t hpin_bytes = 0;
  cudaEvent_t hpin_ev = nullptr;
  int hpin_pending = 0;
  // buffers
  Buf Za, Zb, Zc, Zmap;   // Z2 blocks of the contraction operands, index maps
  Buf Zg;                 // Z2 index maps of the environment Grams and the eigen blocks
  Buf Eb;                 // Z2 blocks of A, W, V for the eigen-solver
  Buf T, T2, Xp, parts, S, Amat, W, V, lam, U64, U32, legres, Y, state, counters, sweeps;
  Buf Ap, Bp, Cb, chA, chB;
  Buf J32, Gns, Vtmp;   // eigen-solver warm start
  // d/d beta carried with T in forward mode (Ising runs; FP64 dense form while on):
  // dT in the slot layout of T, its trace bookkeeping in tstate
  int tangent = 0;
  int is_ising = 0;
  double h = 0.0;
  Buf dT, dT2, dTb, dXp, dS, dA, dU64, eG, eZ, eZt, rank, Yd, tstate;
  Buf dchA, dchB, dchT, dBp, tBp, dCb, tCb;
  Buf dAp, dB64, dU32;   // split-BF16 form: pieces of dT, FP64 staging of dB, dU in FP32
  // tangent == 2: d2T = d^2 T / d beta^2 carried too (FP64 form), and its workspaces
  Buf d2T, d2T2, d2Tb, d2Tc, d2Xp, d2S, d2A, d2U64, eG1, eW, eZ2, eZ2t, d2chA, d2chB, d2Bp, d2Cb, Yd2, parts2;
  // c'-slice shard of a step (hotrg_shard_*): the isometries of (shard_axis, shard_chi)
  // are installed and the new-leg parities derived from them are kept until the
  // gathered new tensor is installed
  int shard_ready = 0;
  int shard_axis = -1, shard_chi = 0;
  int shard_z2 = 0, shard_track = 0;
  double shard_bn_done = 0.0;
  std::vector<unsigned char> shard_par[kMaxD];
  // set while hotrg_graph_capture records steps: no buffer may be (re)allocated and the
  // normalisation takes the step count from the device
  int capturing = 0;
  // launch-shape autotuner of the chain stages (hotrg_set_autotune): stage shape -> CTAs per SM
  int autotune = 0;
  std::map<std::vector<long long>, int> tune_cache;
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
};

namespace {

int dev_alloc(hotrg_ctx* c, Buf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return HOTRG_OK;
  if (c->capturing) return HOTRG_ESTATE;   // a captured step must find its buffers in place
  if (b.p) {
    if (c->ffn) c->ffn(b.p, c->user);
    else cudaFree(b.p);
    c->held -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t want = std::max<size_t>(bytes, 256);
  void* p = nullptr;
  if (c->afn) {
    p = c->afn(want, c->user);
    if (!p) return HOTRG_ENOMEM;
  } else {
    if (cudaMalloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      return HOTRG_ENOMEM;
    }
  }
  b.p = p;
  b.bytes = want;
  c->held += want;
  return HOTRG_OK;
}

void dev_release(hotrg_ctx* c, Buf& b) {
  if (!b.p) return;
  if (c->ffn) c->ffn(b.p, c->user);
  else cudaFree(b.p);
  c->held -= b.bytes;
  b.p = nullptr;
  b.bytes = 0;
}

cudaEvent_t next_event(hotrg_ctx* c) {
  if (c->event_next == c->event_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->event_pool.push_back(e);
  }
  return c->event_pool[c->event_next++];
}

// A chain stage launched with the grid cap (CTAs per SM) the autotuner chose for its shape:
// on the first launch of a shape with autotuning on, each candidate runs once on the real
// operands (a stage writes its output from its inputs, so the runs are idempotent and give
// the same bits), timed with CUDA events; the fastest is kept for the context.  Without
// autotuning, or while a graph is captured, a cached choice is used if there is one, else 16.
template <typename F>
void tuned_chain(hotrg_ctx* c, ChainDesc& cd, int kind, F&& launch) {
  std::vector<long long> key = {kind, cd.total, cd.nn, cd.chi, cd.ndim, cd.a_dim};
  for (int k = 0; k < cd.ndim; ++k) key.push_back(cd.size[k]);
  auto it = c->tune_cache.find(key);
  cd.ctas_per_sm = it != c->tune_cache.end() ? it->second : 16;
  if (!c->autotune || c->capturing || it != c->tune_cache.end()) {
    launch();
    return;
  }
  for (int i = 0; i < 2; ++i)
    if (!c->tune_ev[i]) cudaEventCreate(&c->tune_ev[i]);
  static const int cand[4] = {4, 8, 16, 32};
  float best = 1e30f;
  int choice = 16;
  for (int i = 0; i < 4; ++i) {
    cd.ctas_per_sm = cand[i];
    cudaEventRecord(c->tune_ev[0], c->stream);
    launch();
    cudaEventRecord(c->tune_ev[1], c->stream);
    float ms = 1e30f;
    if (cudaEventSynchronize(c->tune_ev[1]) == cudaSuccess) cudaEventElapsedTime(&ms, c->tune_ev[0], c->tune_ev[1]);
    if (ms < best) {
      best = ms;
      choice = cand[i];
    }
  }
  c->tune_cache[key] = choice;
  cd.ctas_per_sm = choice;
}

// RAII phase mark: records a start/stop event pair on the stream when profiling --
// around every part of a step (profile 1), or around the bottleneck GEMM launches only
// (profile 2, phase 6), kept across steps until hotrg_step_times reads them
struct Phase {
  hotrg_ctx* c;
  int id;
  bool on;
  cudaEvent_t e0 = nullptr;
  Phase(hotrg_ctx* c_, int id_) : c(c_), id(id_), on(c_->profile == 1 || (c_->profile == 2 && id_ == 6)) {
    if (on) {
      e0 = next_event(c);
      cudaEventRecord(e0, c->stream);
    }
  }
  ~Phase() {
    if (on) {
      cudaEvent_t e1 = next_event(c);
      cudaEventRecord(e1, c->stream);
      c->marks.push_back({id, {e0, e1}});
    }
  }
};

#define CHECK_ALLOC(expr)              \
  do {                                 \
    int _r = (expr);                   \
    if (_r != HOTRG_OK) {              \
      c->poisoned = _r;                \
      return _r;                       \
    }                                  \
  } while (0)

// Pinned host buffer of at least `bytes` for an index-map upload; waits for the
// previous upload from it to finish.  nullptr if pinned memory is not available.
void* pinned_stage(hotrg_ctx* c, size_t bytes) {
  if (c->hpin_pending) {
    cudaEventSynchronize(c->hpin_ev);
    c->hpin_pending = 0;
  }
  if (!c->hpin_ev && cudaEventCreateWithFlags(&c->hpin_ev, cudaEventDisableTiming) != cudaSuccess) {
    c->hpin_ev = nullptr;
    return nullptr;
  }
  if (c->hpin_bytes < bytes) {
    if (c->hpin) cudaFreeHost(c->hpin);
    c->hpin = nullptr;
    c->hpin_bytes = 0;
    if (cudaMallocHost(&c->hpin, bytes) != cudaSuccess) {
      cudaGetLastError();
      c->hpin = nullptr;
      return nullptr;
    }
    c->hpin_bytes = bytes;
  }
  return c->hpin;
}

// Jacobi grid-barrier counters: 3 per matrix of one launch (up to 4 (d - 1) parity
// blocks), then 3 for the FP32 warm start
constexpr int kCounters32 = 3 * 4 * kMaxD;
// the FP64 eigen-solver's per-matrix largest squared column norm (16 x 64 bits) after
// the rotation counters of both solvers
constexpr int kColmaxOff = kCounters32 + 4;
constexpr int kCounterInts = kColmaxOff + 2 * 16;

int num_sms() { return sm_count(); }

// A launch wrapper refused its arguments or the launch failed: report which, then the
// CUDA error state (if any) decides the status
int launch_failed(hotrg_ctx* c, const char* what, long long a, long long b, long long k) {
  fprintf(stderr, "hotrg: %s launch failed (%lld, %lld, %lld)\n", what, a, b, k);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) fprintf(stderr, "hotrg: CUDA error %s\n", cudaGetErrorString(e));
  c->poisoned = HOTRG_ECUDA;
  return HOTRG_ECUDA;
}

// A launch error left pending by the kernels of one part of the step: report the part
int pending_error(hotrg_ctx* c, const char* part) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return HOTRG_OK;
  fprintf(stderr, "hotrg: CUDA error after %s: %s\n", part, cudaGetErrorString(e));
  c->poisoned = HOTRG_ECUDA;
  return HOTRG_ECUDA;
}

int cuda_status(hotrg_ctx* c) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "hotrg: CUDA error %s\n", cudaGetErrorString(e));
    c->poisoned = HOTRG_ECUDA;
    return HOTRG_ECUDA;
  }
  return HOTRG_OK;
}

// strides of the slot layout for bond dims per slot
void slot_strides(int d, const int* slot_chi, long long* row_stride, long long* col_stride,
                  long long* R) {
  long long r = 1;
  for (int s = 0; s < d; ++s) r *= slot_chi[s];
  *R = r;
  long long st = 1;
  for (int s = d - 1; s >= 0; --s) {
    col_stride[s] = st;
    row_stride[s] = st * r;
    st *= slot_chi[s];
  }
}

// Permute T (slot layout with `from` order) into slot layout with `to` order.
void permute_slots(hotrg_ctx* c, const double* in, const int* from, double* out, const int* to,
                   double scale) {
  int d = c->d;
  int chi_from[kMaxD], chi_to[kMaxD];
  for (int s = 0; s < d; ++s) {
    chi_from[s] = c->chis[from[s]];
    chi_to[s] = c->chis[to[s]];
  }
  long long rs[kMaxD], cs[kMaxD], R;
  slot_strides(d, chi_from, rs, cs, &R);
  long long size[kMaxDims], ist[kMaxDims];
  for (int s = 0; s < d; ++s) {
    int src = 0;
    for (int t = 0; t < d; ++t)
      if (from[t] == to[s]) src = t;
    size[s] = chi_to[s];
    ist[s] = rs[src];
    size[d + s] = chi_to[s];
    ist[d + s] = cs[src];
  }
  launch_permute(in, out, 2 * d, size, ist, scale, c->stream);
}

// interchange layout (x_0, x_0', x_1, x_1', ...) <-> slot layout
void interchange_to_slots(hotrg_ctx* c, const double* in, double* out) {
  int d = c->d;
  // input strides of the interchange layout
  long long st[2 * kMaxD];
  long long acc = 1;
  for (int k = 2 * d - 1; k >= 0; --k) {
    st[k] = acc;
    acc *= c->chis[k / 2];
  }
  long long size[kMaxDims], ist[kMaxDims];
  for (int s = 0; s < d; ++s) {
    int ax = c->order[s];
    size[s] = c->chis[ax];
    ist[s] = st[2 * ax];
    size[d + s] = c->chis[ax];
    ist[d + s] = st[2 * ax + 1];
  }
  launch_permute(in, out, 2 * d, size, ist, 1.0, c->stream);
}

void slots_to_interchange(hotrg_ctx* c, const double* in, double* out) {
  int d = c->d;
  int slot_chi[kMaxD];
  for (int s = 0; s < d; ++s) slot_chi[s] = c->chis[c->order[s]];
  long long rs[kMaxD], cs[kMaxD], R;
  slot_strides(d, slot_chi, rs, cs, &R);
  long long size[kMaxDims], ist[kMaxDims];
  for (int k = 0; k < d; ++k) {
    int s = 0;
    for (int t = 0; t < d; ++t)
      if (c->order[t] == k) s = t;
    size[2 * k] = c->chis[k];
    ist[2 * k] = rs[s];
    size[2 * k + 1] = c->chis[k];
    ist[2 * k + 1] = cs[s];
  }
  launch_permute(in, out, 2 * d, size, ist, 1.0, c->stream);
}

long long tensor_elems(hotrg_ctx* c) {
  long long n = 1;
  for (int k = 0; k < c->d; ++k) n *= (long long)c->chis[k] * c->chis[k];
  return n;
}

// Trace, Y, X and the ln Z bookkeeping of the tensor in c->T (slot layout),
// then normalisation of c->T in place (Secs. 4.2.1 / 4.2.11-4.2.16).
void trace_and_normalise(hotrg_ctx* c, double* Tsrc, int first) {
  int d = c->d;
  int chi_c = c->chis[c->order[0]];
  long long pn = 1;
  for (int s = 1; s < d; ++s) pn *= c->chis[c->order[s]];
  DevState* st = (DevState*)c->state.p;
  launch_trace_y(Tsrc, chi_c, pn, (double*)c->Y.p, c->stream);
  launch_finish_step((double*)c->Y.p, chi_c, st, c->capturing ? -1 : c->p, first, c->stream);
  launch_scale(Tsrc, (double*)c->T.p, tensor_elems(c), st, c->stream);
}

// The same for the derivative dTsrc of the new, unnormalised tensor, after
// trace_and_normalise has run: d ln Tr, the d/d beta of the ln Z bookkeeping, and
// c->dT = d(T / Tr T) = dTsrc / Tr T - (d ln Tr) c->T.
void tangent_trace_and_normalise(hotrg_ctx* c, const double* dTsrc, int first) {
  int d = c->d;
  int chi_c = c->chis[c->order[0]];
  long long pn = 1;
  for (int s = 1; s < d; ++s) pn *= c->chis[c->order[s]];
  const DevState* st = (const DevState*)c->state.p;
  TanState* tst = (TanState*)c->tstate.p;
  launch_trace_y(dTsrc, chi_c, pn, (double*)c->Yd.p, c->stream);
  launch_finish_tangent((const double*)c->Yd.p, chi_c, st, tst, c->p, first, c->stream);
  launch_tangent_scale(dTsrc, (const double*)c->T.p, (double*)c->dT.p, tensor_elems(c), st, tst, c->stream);
}

// The second order, after tangent_trace_and_normalise has run: d2 ln Tr, the d^2/d beta^2
// of the ln Z bookkeeping, and c->d2T = d^2(T / Tr T) from d2Tsrc and dTsrc of the new,
// unnormalised tensor and the normalised c->dT, c->T.
void tangent2_trace_and_normalise(hotrg_ctx* c, const double* d2Tsrc, const double* dTsrc, int first) {
  int d = c->d;
  int chi_c = c->chis[c->order[0]];
  long long pn = 1;
  for (int s = 1; s < d; ++s) pn *= c->chis[c->order[s]];
  const DevState* st = (const DevState*)c->state.p;
  TanState* tst = (TanState*)c->tstate.p;
  launch_trace_y(d2Tsrc, chi_c, pn, (double*)c->Yd2.p, c->stream);
  launch_finish_tangent2((const double*)c->Yd2.p, chi_c, st, tst, c->p, first, c->stream);
  launch_tangent2_scale(d2Tsrc, dTsrc, (const double*)c->dT.p, (const double*)c->T.p, (double*)c->d2T.p,
                        tensor_elems(c), st, tst, c->stream);
}

int start_run(hotrg_ctx* c) {
  CHECK_ALLOC(dev_alloc(c, c->state, sizeof(DevState)));
  CHECK_ALLOC(dev_alloc(c, c->Y, sizeof(double) * kMaxBond * kMaxBond));
  cudaMemsetAsync(c->state.p, 0, sizeof(DevState), c->stream);
  trace_and_normalise(c, (double*)c->T.p, 1);
  return cuda_status(c);
}

int sync_and_status(hotrg_ctx* c, DevState* out) {
  if (c->poisoned) return HOTRG_ESTATE;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    c->poisoned = HOTRG_ECUDA;
    return HOTRG_ECUDA;
  }
  DevState st;
  if (cudaMemcpy(&st, c->state.p, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    c->poisoned = HOTRG_ECUDA;
    return HOTRG_ECUDA;
  }
  if (st.status != 0) {
    c->poisoned = st.status;
    return st.status;
  }
  if (out) *out = st;
  return HOTRG_OK;
}

}  // namespace

extern "C" {

const char* hotrg_strerror(int status) {
  switch (status) {
    case HOTRG_OK: return "ok";
    case HOTRG_EINVAL: return "invalid argument";
    case HOTRG_ENOMEM: return "device allocation failed";
    case HOTRG_ECUDA: return "CUDA call failed";
    case HOTRG_ENUMERIC: return "trace of the new tensor is not positive and finite";
    case HOTRG_ENOTCONV: return "Jacobi eigen-solver hit its sweep cap";
    case HOTRG_ETIMEOUT: return "bounded device wait expired";
    case HOTRG_ESTATE: return "context unusable (earlier failure) or no step yet";
    default: return "unknown status";
  }
}

int hotrg_init_ising(int d, double beta, double h, hotrg_ctx** out) {
  if (!out || d < 2 || d > kMaxD || !(beta >= 0.0) || !std::isfinite(beta) || !std::isfinite(h))
    return HOTRG_EINVAL;
  *out = nullptr;
  hotrg_ctx* c = new hotrg_ctx();
  c->d = d;
  c->beta = beta;
  c->h = h;
  c->is_ising = 1;
  for (int k = 0; k < d; ++k) {
    c->chis[k] = 2;
    c->order[k] = k;
    c->par[k] = {0, 1};   // index 0 carries sqrt(cosh), index 1 sigma sqrt(sinh): even, odd
  }
  // at h = 0 every element of odd total parity vanishes (spin-flip symmetry)
  c->z2_valid = h == 0.0 ? 1 : 0;
  int r = dev_alloc(c, c->T, sizeof(double) << (2 * d));
  if (r == HOTRG_OK) {
    launch_init_ising((double*)c->T.p, d, beta, h, c->stream);
    r = start_run(c);
  }
  if (r != HOTRG_OK) {
    hotrg_free(c);
    return r;
  }
  *out = c;
  return HOTRG_OK;
}

int hotrg_init_tensor(int d, const int* chis, const double* T, double beta, hotrg_ctx** out) {
  if (!out || !chis || !T || d < 2 || d > kMaxD || !(beta >= 0.0)) return HOTRG_EINVAL;
  for (int k = 0; k < d; ++k)
    if (chis[k] < 1 || chis[k] > 32) return HOTRG_EINVAL;
  *out = nullptr;
  hotrg_ctx* c = new hotrg_ctx();
  c->d = d;
  c->beta = beta;
  for (int k = 0; k < d; ++k) {
    c->chis[k] = chis[k];
    c->order[k] = k;
  }
  size_t bytes = sizeof(double) * tensor_elems(c);
  int r = dev_alloc(c, c->T, bytes);
  if (r == HOTRG_OK) r = dev_alloc(c, c->Xp, bytes);
  if (r == HOTRG_OK) {
    if (cudaMemcpyAsync(c->Xp.p, T, bytes, cudaMemcpyDefault, c->stream) != cudaSuccess) r = HOTRG_ECUDA;
  }
  if (r == HOTRG_OK) {
    interchange_to_slots(c, (const double*)c->Xp.p, (double*)c->T.p);
    r = start_run(c);
  }
  if (r != HOTRG_OK) {
    cudaGetLastError();
    hotrg_free(c);
    return r;
  }
  *out = c;
  return HOTRG_OK;
}

int hotrg_set_tensor(hotrg_ctx* c, const int* chis, const double* T) {
  if (!c || !chis || !T) return HOTRG_EINVAL;
  if (c->poisoned) return HOTRG_ESTATE;
  for (int k = 0; k < c->d; ++k)
    if (chis[k] < 1 || chis[k] > 32) return HOTRG_EINVAL;
  for (int k = 0; k < c->d; ++k) {
    c->chis[k] = chis[k];
    c->order[k] = k;
  }
  size_t bytes = sizeof(double) * tensor_elems(c);
  CHECK_ALLOC(dev_alloc(c, c->T, bytes));
  CHECK_ALLOC(dev_alloc(c, c->Xp, bytes));
  if (cudaMemcpyAsync(c->Xp.p, T, bytes, cudaMemcpyDefault, c->stream) != cudaSuccess)
    return cuda_status(c);
  interchange_to_slots(c, (const double*)c->Xp.p, (double*)c->T.p);
  c->last_valid = 0;
  c->z2_valid = 0;   // until hotrg_set_parity declares and checks the parities
  c->tangent = 0;    // the derivative of a tensor set from outside is not known
  int r = cuda_status(c);
  if (r != HOTRG_OK) return r;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_status(c);
  return HOTRG_OK;
}

int hotrg_set_stream(hotrg_ctx* c, void* stream) {
  if (!c) return HOTRG_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_status(c);
  c->stream = (cudaStream_t)stream;
  return HOTRG_OK;
}

int hotrg_set_allocator(hotrg_ctx* c, hotrg_alloc_fn alloc, hotrg_free_fn free_fn, void* user) {
  if (!c || (!alloc) != (!free_fn)) return HOTRG_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_status(c);
  // keep the tensor and the run state (and their derivatives), drop every workspace
  Buf keep[5] = {c->T, c->state, c->dT, c->tstate, c->d2T};
  size_t keep_bytes[5] = {c->T.bytes, c->state.bytes, c->tangent ? c->dT.bytes : 0,
                          c->tangent ? c->tstate.bytes : 0, c->tangent == 2 ? c->d2T.bytes : 0};
  std::vector<char> host[5];
  for (int i = 0; i < 5; ++i) {
    host[i].resize(keep_bytes[i]);
    if (keep_bytes[i] && keep[i].p &&
        cudaMemcpy(host[i].data(), keep[i].p, keep_bytes[i], cudaMemcpyDeviceToHost) != cudaSuccess)
      return cuda_status(c);
  }
  int n = 0;
  Buf* b[] = {&c->T,  &c->T2, &c->Xp,     &c->parts, &c->S,     &c->Amat,     &c->W,
              &c->V,  &c->lam, &c->U64,   &c->U32,   &c->legres, &c->Y,       &c->state,
              &c->counters, &c->sweeps, &c->Ap, &c->Bp, &c->Cb, &c->chA, &c->chB,
              &c->J32,  &c->Gns, &c->Vtmp, &c->Za, &c->Zb, &c->Zc, &c->Zmap, &c->Zg, &c->Eb,
              &c->dT, &c->dT2, &c->dTb, &c->dXp, &c->dS, &c->dA, &c->dU64, &c->eG, &c->eZ, &c->eZt,
              &c->rank, &c->Yd, &c->tstate, &c->dchA, &c->dchB, &c->dchT, &c->dBp, &c->tBp, &c->dCb,
              &c->tCb, &c->dAp, &c->dB64, &c->dU32, &c->d2T, &c->d2T2, &c->d2Tb, &c->d2Tc, &c->d2Xp,
              &c->d2S, &c->d2A, &c->d2U64, &c->eG1, &c->eW, &c->eZ2, &c->eZ2t, &c->d2chA, &c->d2chB,
              &c->d2Bp, &c->d2Cb, &c->Yd2, &c->parts2};
  n = (int)(sizeof(b) / sizeof(b[0]));
  for (int i = 0; i < n; ++i) dev_release(c, *b[i]);
  c->afn = alloc;
  c->ffn = free_fn;
  c->user = user;
  c->last_valid = 0;
  Buf* kb[5] = {&c->T, &c->state, &c->dT, &c->tstate, &c->d2T};
  for (int i = 0; i < 5; ++i) {
    if (!keep_bytes[i]) continue;
    CHECK_ALLOC(dev_alloc(c, *kb[i], keep_bytes[i]));
    if (cudaMemcpy(kb[i]->p, host[i].data(), keep_bytes[i], cudaMemcpyHostToDevice) != cudaSuccess)
      return cuda_status(c);
  }
  CHECK_ALLOC(dev_alloc(c, c->Y, sizeof(double) * kMaxBond * kMaxBond));
  if (c->tangent) CHECK_ALLOC(dev_alloc(c, c->Yd, sizeof(double) * kMaxBond * kMaxBond));
  if (c->tangent == 2) CHECK_ALLOC(dev_alloc(c, c->Yd2, sizeof(double) * kMaxBond * kMaxBond));
  return HOTRG_OK;
}

int hotrg_set_autotune(hotrg_ctx* c, int enable) {
  if (!c || enable < 0 || enable > 1) return HOTRG_EINVAL;
  c->autotune = enable;
  return HOTRG_OK;
}

int hotrg_autotune_entries(hotrg_ctx* c, int* n, int* choices, int cap) {
  if (!c || !n) return HOTRG_EINVAL;
  *n = (int)c->tune_cache.size();
  if (!choices) return HOTRG_OK;
  if (cap < *n) return HOTRG_EINVAL;
  int i = 0;
  for (const auto& kv : c->tune_cache) choices[i++] = kv.second;
  return HOTRG_OK;
}

int hotrg_set_precision(hotrg_ctx* c, int mode) {
  if (!c || mode < HOTRG_PREC_FP64 || mode > HOTRG_PREC_TF32X3) return HOTRG_EINVAL;
  if (c->tangent == 2 && mode != HOTRG_PREC_FP64) return HOTRG_EINVAL;   // second order: FP64 form
  if (mode != HOTRG_PREC_FP64 && !tc_gemm_ready()) return HOTRG_ECUDA;
  c->precision = mode;
  return HOTRG_OK;
}

namespace {

// One phase of a step split over ranks by c'-slices (hotrg_shard_*).  PH_FULL is
// the whole step of one process.
enum ShardPhase { PH_FULL = 0, PH_ENV = 1, PH_ISO = 2, PH_CONTRACT = 3, PH_FINISH = 4 };
struct Shard {
  int phase = PH_FULL;
  int part = 0, nparts = 1;      // PH_ENV: this rank's share of each Gram's summed index
  int c_lo = 0, c_hi = 0;        // PH_CONTRACT: the c'-slices [c_lo, c_hi)
  double* out = nullptr;         // PH_ENV: partial Grams; PH_CONTRACT: slices
  int64_t cap = 0;
  int64_t* n_out = nullptr;
  const double* in = nullptr;    // PH_ISO: summed Grams; PH_FINISH: every slice
};

int step_impl(hotrg_ctx* c, int axis, int chi, const Shard& sh);

}  // namespace

int hotrg_step(hotrg_ctx* c, int axis, int chi) { return step_impl(c, axis, chi, Shard()); }

namespace {

int step_impl(hotrg_ctx* c, int axis, int chi, const Shard& sh) {
  if (!c) return HOTRG_EINVAL;
  if (c->poisoned) return HOTRG_ESTATE;
  const int d = c->d;
  if (axis < 0 || axis >= d || chi < 1 || chi > 32) return HOTRG_EINVAL;
  const int phase = sh.phase;
  if (phase != PH_FULL && c->tangent) return HOTRG_EINVAL;   // the shard carries no derivative
  if ((phase == PH_CONTRACT || phase == PH_FINISH) &&
      (!c->shard_ready || c->shard_axis != axis || c->shard_chi != chi))
    return HOTRG_ESTATE;
  if (phase == PH_FULL || phase == PH_ENV) c->shard_ready = 0;
  cudaStream_t s = c->stream;

  // ---- slot order for this step: Current = axis, Next j = (axis + j) mod d
  int to[kMaxD];
  for (int k = 0; k < d; ++k) to[k] = (axis + k) % d;
  const int chi_c = c->chis[axis];
  int chij[kMaxD], nnew[kMaxD];
  long long P = 1, Pn = 1;
  for (int j = 1; j < d; ++j) {
    chij[j] = c->chis[to[j]];
    nnew[j] = std::min(chij[j] * chij[j], chi);
    P *= chij[j];
    Pn *= nnew[j];
  }
  const long long R = (long long)chi_c * P;      // rows = cols of T
  const long long Rn = (long long)chi_c * Pn;    // rows = cols of T'
  const long long RR = R * R;
  // bottleneck work of this step: 2 * R^2 * (P_new P) per c'-slice, chi_c slices
  const double bn_flops = 2.0 * (double)R * (double)R * (double)Pn * (double)P * (double)chi_c;
  // the derivative d/d beta, when carried, runs with the dense contraction
  const bool tangent = c->tangent != 0;
  const bool tan2 = c->tangent == 2;   // d^2 / d beta^2 carried too (FP64 form)
  const bool fp64 = c->precision == HOTRG_PREC_FP64 || bn_flops < c->fp64_below;
  if (tan2 && !fp64) return HOTRG_EINVAL;
  c->last_fp64 = fp64 ? 1 : 0;

  if (c->profile != 2) {   // profile 2 keeps the marks of several steps
    c->marks.clear();
    c->event_next = 0;
  }
  CHECK_ALLOC(dev_alloc(c, c->T2, sizeof(double) * RR));
  CHECK_ALLOC(dev_alloc(c, c->Xp, sizeof(double) * RR));
  bool same = true;
  for (int k = 0; k < d; ++k) same = same && (c->order[k] == to[k]);
  double* Tc = (double*)c->T.p;
  if (!same) {
    Phase ph(c, 0);
    permute_slots(c, (const double*)c->T.p, c->order, (double*)c->T2.p, to, 1.0);
    std::swap(c->T, c->T2);
    if (tangent) {
      CHECK_ALLOC(dev_alloc(c, c->dT2, sizeof(double) * RR));
      permute_slots(c, (const double*)c->dT.p, c->order, (double*)c->dT2.p, to, 1.0);
      std::swap(c->dT, c->dT2);
    }
    if (tan2) {
      CHECK_ALLOC(dev_alloc(c, c->d2T2, sizeof(double) * RR));
      permute_slots(c, (const double*)c->d2T.p, c->order, (double*)c->d2T2.p, to, 1.0);
      std::swap(c->d2T, c->d2T2);
    }
    Tc = (double*)c->T.p;
    for (int k = 0; k < d; ++k) c->order[k] = to[k];
  }

  // strides of T in slot layout
  long long rs[kMaxD], cs[kMaxD], Rchk;
  {
    int sc[kMaxD];
    for (int k = 0; k < d; ++k) sc[k] = c->chis[to[k]];
    slot_strides(d, sc, rs, cs, &Rchk);
  }

  // ---- environments (Sec. 3.2; Sec. 4.2.4), FP64
  // legs grouped by n = chi_j^2 so that one Jacobi launch covers a group
  const int nlegs = d - 1;
  int grp_of[kMaxD], grp_n[kMaxD], grp_first_mat[kMaxD], ngrp = 0, mat_of_leg[kMaxD];
  {
    int nmat_acc = 0;
    for (int j = 1; j < d; ++j) {
      int n = chij[j] * chij[j];
      int g = -1;
      for (int q = 0; q < ngrp; ++q)
        if (grp_n[q] == n) g = q;
      if (g < 0) {
        g = ngrp++;
        grp_n[g] = n;
      }
      grp_of[j] = g;
    }
    // matrices laid out group by group, two per leg (A, A')
    for (int g = 0; g < ngrp; ++g) {
      grp_first_mat[g] = nmat_acc;
      for (int j = 1; j < d; ++j)
        if (grp_of[j] == g) {
          mat_of_leg[j] = nmat_acc;
          nmat_acc += 2;
        }
    }
  }
  // matrix element offsets: group base + local index * n^2
  long long mat_elem_off[2 * kMaxD];
  long long total_mat_elems = 0;
  {
    for (int g = 0; g < ngrp; ++g) {
      int cnt = 0;
      for (int j = 1; j < d; ++j)
        if (grp_of[j] == g) cnt += 2;
      for (int j = 1; j < d; ++j)
        if (grp_of[j] == g) {
          int local = mat_of_leg[j] - grp_first_mat[g];
          mat_elem_off[2 * j] = total_mat_elems + (long long)local * grp_n[g] * grp_n[g];
          mat_elem_off[2 * j + 1] = mat_elem_off[2 * j] + (long long)grp_n[g] * grp_n[g];
        }
      total_mat_elems += (long long)cnt * grp_n[g] * grp_n[g];
    }
  }
  long long mmax = 0, nmax = 0;
  for (int j = 1; j < d; ++j) {
    mmax = std::max<long long>(mmax, (long long)chij[j] * chi_c);
    nmax = std::max<long long>(nmax, (long long)chij[j] * chij[j]);
  }
  const int nsplit_max = 256;
  // split-K count of a Gram (upper tiles of an m x m product over K): the CTAs that share
  // an SM share its FP64 units, so the step lasts as long as the busiest SM's K-work.
  // Among the splits that give at least two CTAs per SM (to hide latency; fewer only if
  // K is too short), pick the one that minimises (CTAs on the busiest SM) x (K per CTA
  // + a fixed cost).
  auto gram_splits = [&](long long m, long long K) {
    const long long tl = gram_tile();
    const long long ut = ((m + tl - 1) / tl) * ((m + tl - 1) / tl + 1) / 2;
    const long long sms = num_sms();
    int best = 1, best_any = 1;
    double best_cost = 1e300, best_any_cost = 1e300;
    for (int ns = 1; ns <= nsplit_max; ++ns) {
      long long kchunk = (K + ns - 1) / ns;
      kchunk = (kchunk + 15) / 16 * 16;
      if (kchunk < 64 && ns > 1) break;
      const long long used = (K + kchunk - 1) / kchunk;
      const double cost = (double)((ut * used + sms - 1) / sms) * (double)(kchunk + 64);
      if (cost < best_any_cost * 0.999) {
        best_any_cost = cost;
        best_any = ns;
      }
      if (ut * used >= 2 * sms && cost < best_cost * 0.999) {
        best_cost = cost;
        best = ns;
      }
    }
    return best_cost < 1e300 ? best : best_any;
  };
  CHECK_ALLOC(dev_alloc(c, c->parts, sizeof(double) * nsplit_max * mmax * mmax));
  CHECK_ALLOC(dev_alloc(c, c->S, sizeof(double) * 4 * nlegs * mmax * mmax));
  CHECK_ALLOC(dev_alloc(c, c->Amat, sizeof(double) * total_mat_elems));
  CHECK_ALLOC(dev_alloc(c, c->W, sizeof(double) * total_mat_elems));
  CHECK_ALLOC(dev_alloc(c, c->V, sizeof(double) * total_mat_elems));
  CHECK_ALLOC(dev_alloc(c, c->J32, sizeof(float) * 2 * total_mat_elems));
  CHECK_ALLOC(dev_alloc(c, c->Gns, sizeof(double) * total_mat_elems));
  CHECK_ALLOC(dev_alloc(c, c->Vtmp, sizeof(double) * total_mat_elems));
  CHECK_ALLOC(dev_alloc(c, c->counters, sizeof(int) * kCounterInts));
  CHECK_ALLOC(dev_alloc(c, c->sweeps, sizeof(int) * 6 * kMaxD));

  // Gram of leg j, kind: X = T with the free pair (n_j or n'_j, c' or c) first, rest after
  // kind 0: S^  free (n_j, c');  1: S~  free (n_j, c);
  // kind 2: S^' free (n'_j, c'); 3: S~' free (n'_j, c)
  auto gram_dims = [&](int j, int kind, long long* size, long long* ist, int* pslot) {
    const int fpos = (kind < 2) ? j : d + j;
    const int cpos = (kind == 0 || kind == 2) ? d : 0;
    int nd = 0;
    size[nd] = chij[j];
    pslot[nd] = j;
    ist[nd++] = fpos < d ? rs[fpos] : cs[fpos - d];
    size[nd] = chi_c;
    pslot[nd] = 0;
    ist[nd++] = cpos < d ? rs[cpos] : cs[cpos - d];
    for (int q = 0; q < 2 * d; ++q) {
      if (q == fpos || q == cpos) continue;
      size[nd] = q < d ? c->chis[to[q]] : c->chis[to[q - d]];
      pslot[nd] = q % d;
      ist[nd++] = q < d ? rs[q] : cs[q - d];
    }
    return nd;
  };
  // Z2 blocks of the Grams: the rows (free pair) and the summed index, both listed even
  // parity first, as element offsets into T; per leg the block and position of each row
  const bool z2g = c->z2_valid && c->z2_enabled && c->tangent != 2;
  const bool env_phase = phase == PH_FULL || phase == PH_ENV || phase == PH_ISO;
  long long gz_roff[kMaxD][4], gz_koff[kMaxD][4], gz_rowmap[kMaxD];
  long long gz_mb[kMaxD][2], gz_Kb[kMaxD][4][2], gz_n64 = 0, gz_eig[kMaxD];
  int eig_nb[kMaxD][2];
  if (z2g && env_phase) {
    long long n64 = 0, n32 = 0;
    for (int j = 1; j < d; ++j) {
      const long long m = (long long)chij[j] * chi_c;
      for (int kind = 0; kind < 4; ++kind) {
        gz_roff[j][kind] = n64;
        gz_koff[j][kind] = n64 + m;
        n64 += m + RR / m;
      }
      gz_rowmap[j] = n32;
      n32 += 2 * m;
      gz_eig[j] = n32;                       // rows by parity, block, position (n = chi_j^2)
      n32 += 3LL * chij[j] * chij[j];
    }
    gz_n64 = n64;   // the int maps follow the offsets
    const size_t bytes = sizeof(long long) * n64 + sizeof(int) * n32;
    long long* h64 = (long long*)pinned_stage(c, bytes);
    std::vector<long long> h64v;
    if (!h64) {
      h64v.resize((bytes + 7) / 8);
      h64 = h64v.data();
    }
    int* h32 = (int*)(h64 + n64);
    std::vector<long long> offs;
    std::vector<unsigned char> pk;
    for (int j = 1; j < d; ++j) {
      const std::vector<unsigned char>& pf = c->par[to[j]];
      const std::vector<unsigned char>& pc = c->par[to[0]];
      int* blk = h32 + gz_rowmap[j];
      int* pos = blk + (long long)chij[j] * chi_c;
      long long cnt[2] = {0, 0};
      for (int f = 0; f < chij[j]; ++f)
        for (int cu = 0; cu < chi_c; ++cu) {
          const int b = pf[f] ^ pc[cu];
          blk[f * chi_c + cu] = b;
          pos[f * chi_c + cu] = (int)cnt[b]++;
        }
      gz_mb[j][0] = cnt[0];
      gz_mb[j][1] = cnt[1];
      {
        // composite index r = hat + check chi_j of A^(j): parity pf[hat] ^ pf[check]
        const int cj = chij[j], n = cj * cj;
        int* rows = h32 + gz_eig[j];
        int* eb = rows + n;
        int* ep = eb + n;
        int ec[2] = {0, 0};
        for (int r = 0; r < n; ++r) {
          const int b = pf[r % cj] ^ pf[r / cj];
          eb[r] = b;
          ep[r] = ec[b]++;
        }
        int w2[2] = {0, ec[0]};
        for (int r = 0; r < n; ++r) rows[w2[eb[r]]++] = r;
        eig_nb[j][0] = ec[0];
        eig_nb[j][1] = ec[1];
      }
      for (int kind = 0; kind < 4; ++kind) {
        long long size[kMaxDims], ist[kMaxDims];
        int pslot[kMaxDims];
        const int nd = gram_dims(j, kind, size, ist, pslot);
        long long* ro = h64 + gz_roff[j][kind];
        long long w[2] = {0, cnt[0]};
        for (int f = 0; f < chij[j]; ++f)
          for (int cu = 0; cu < chi_c; ++cu) ro[w[pf[f] ^ pc[cu]]++] = f * ist[0] + cu * ist[1];
        // the summed index, row-major over dims 2 .. nd-1, by an odometer
        const long long K = RR / ((long long)chij[j] * chi_c);
        offs.resize(K);
        pk.resize(K);
        long long idx[kMaxDims] = {0};
        long long off = 0;
        int par_ = 0;
        for (int q = 2; q < nd; ++q) par_ ^= c->par[to[pslot[q]]][0];
        long long kc[2] = {0, 0};
        for (long long k = 0; k < K; ++k) {
          offs[k] = off;
          pk[k] = (unsigned char)par_;
          ++kc[par_];
          for (int q = nd - 1; q >= 2; --q) {
            const std::vector<unsigned char>& pq = c->par[to[pslot[q]]];
            par_ ^= pq[idx[q]];
            off -= idx[q] * ist[q];
            if (++idx[q] < size[q]) {
              par_ ^= pq[idx[q]];
              off += idx[q] * ist[q];
              break;
            }
            idx[q] = 0;
            par_ ^= pq[0];
          }
        }
        long long* ko = h64 + gz_koff[j][kind];
        long long wk[2] = {0, kc[0]};
        for (long long k = 0; k < K; ++k) ko[wk[pk[k]]++] = offs[k];
        gz_Kb[j][kind][0] = kc[0];
        gz_Kb[j][kind][1] = kc[1];
      }
    }
    CHECK_ALLOC(dev_alloc(c, c->Zg, bytes));
    if (cudaMemcpyAsync(c->Zg.p, h64, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return cuda_status(c) == HOTRG_OK ? (c->poisoned = HOTRG_ECUDA) : HOTRG_ECUDA;
    if (h64v.empty()) {
      cudaEventRecord(c->hpin_ev, s);
      c->hpin_pending = 1;
    }
  }
  // the shard's layout of the Grams: legs j = 1 .. d-1, kinds 0 .. 3, each m_j x m_j
  // row-major (m_j = chi_j chi_c), concatenated
  long long shard_s_elems = 0;
  for (int j = 1; j < d; ++j) shard_s_elems += 4LL * chij[j] * chi_c * chij[j] * chi_c;
  if (phase == PH_ENV || phase == PH_ISO) {
    if (sh.n_out) *sh.n_out = shard_s_elems;
    if ((phase == PH_ENV && (!sh.out || sh.cap < shard_s_elems)) ||
        (phase == PH_ISO && (!sh.in || sh.cap != shard_s_elems)))
      return HOTRG_EINVAL;
  }
  for (int j = 1; j < d && env_phase; ++j) {
    Phase ph(c, 1);
    const long long m = (long long)chij[j] * chi_c;
    const long long K = RR / m;
    for (int kind = 0; kind < 4; ++kind) {
      long long size[kMaxDims], ist[kMaxDims];
      int pslot[kMaxDims];
      const int nd = gram_dims(j, kind, size, ist, pslot);
      double* Sdst = (double*)c->S.p + ((long long)(j - 1) * 4 + kind) * mmax * mmax;
      if (phase == PH_ISO) continue;   // the summed Grams are installed below
      // PH_ENV: this rank's part of the summed index (of each parity block)
      auto kpart = [&](long long kk, long long* lo) {
        *lo = kk * sh.part / sh.nparts;
        return kk * (sh.part + 1) / sh.nparts - *lo;
      };
      if (z2g) {
        const long long* zg = (const long long*)c->Zg.p;
        double* X = (double*)c->Xp.p;
        launch_z2_gather_rc(Tc, zg + gz_roff[j][kind], (int)m, zg + gz_koff[j][kind], K, X, s);
        const double* pb[2] = {(const double*)c->parts.p, (const double*)c->parts.p};
        int nsb[2] = {0, 0};
        long long poff = 0;
        for (int b = 0; b < 2; ++b) {
          const long long mb = gz_mb[j][b];
          long long Kb = gz_Kb[j][kind][b];
          const long long r0 = b == 0 ? 0 : gz_mb[j][0];
          long long k0 = b == 0 ? 0 : gz_Kb[j][kind][0];
          if (phase == PH_ENV) {
            long long lo = 0;
            Kb = kpart(Kb, &lo);
            k0 += lo;
          }
          if (mb == 0 || Kb == 0) continue;
          const int nsplit = gram_splits(mb, Kb);
          double* pdst = (double*)c->parts.p + poff;
          nsb[b] = launch_gemm_nt_f64(X + r0 * K + k0, K, X + r0 * K + k0, K, pdst, mb, mb * mb, (int)mb,
                                      (int)mb, Kb, nsplit, 1, s);
          pb[b] = pdst;
          poff += (long long)nsb[b] * mb * mb;
        }
        const int* zi = (const int*)(zg + gz_n64) + gz_rowmap[j];
        launch_z2_reduce_sym(pb[0], nsb[0], (int)gz_mb[j][0], pb[1], nsb[1], (int)gz_mb[j][1], zi,
                             zi + m, (int)m, Sdst, s);
        continue;
      }
      launch_permute(Tc, (double*)c->Xp.p, nd, size, ist, 1.0, s);
      long long k_lo = 0, Kp = K;
      if (phase == PH_ENV) Kp = kpart(K, &k_lo);
      if (Kp == 0) {
        cudaMemsetAsync(Sdst, 0, sizeof(double) * m * m, s);
        continue;
      }
      const int nsplit = gram_splits(m, Kp);
      // the GEMM may round nsplit down: reduce the partials it wrote
      const double* X0 = (const double*)c->Xp.p + k_lo;
      const int used = launch_gemm_nt_f64(X0, K, X0, K, (double*)c->parts.p, m, m * m, (int)m, (int)m, Kp,
                                          nsplit, 1, s);
      launch_reduce_sym((const double*)c->parts.p, used, (int)m, Sdst, s);
    }
    double* S0 = (double*)c->S.p + ((long long)(j - 1) * 4) * mmax * mmax;
    if (phase == PH_ENV || phase == PH_ISO) {
      // out: this rank's partial Grams; in: the Grams summed over the ranks
      const long long mm = m * m;
      long long off = 0;
      for (int q = 1; q < j; ++q) off += 4LL * chij[q] * chi_c * chij[q] * chi_c;
      for (int kind = 0; kind < 4; ++kind) {
        double* Sk = S0 + kind * mmax * mmax;
        const cudaError_t ce =
            phase == PH_ENV
                ? cudaMemcpyAsync(sh.out + off + kind * mm, Sk, sizeof(double) * mm, cudaMemcpyDefault, s)
                : cudaMemcpyAsync(Sk, sh.in + off + kind * mm, sizeof(double) * mm, cudaMemcpyDefault, s);
        if (ce != cudaSuccess) return cuda_status(c) == HOTRG_OK ? (c->poisoned = HOTRG_ECUDA) : HOTRG_ECUDA;
      }
      if (phase == PH_ENV) continue;
    }
    launch_assemble_a(S0, S0 + mmax * mmax, chij[j], chi_c, (double*)c->Amat.p + mat_elem_off[2 * j], s);
    launch_assemble_a(S0 + 2 * mmax * mmax, S0 + 3 * mmax * mmax, chij[j], chi_c,
                      (double*)c->Amat.p + mat_elem_off[2 * j + 1], s);
  }
  if (phase == PH_ENV) {
    if (pending_error(c, "the environments") != HOTRG_OK) return HOTRG_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_status(c);
    return cuda_status(c);
  }

  if (pending_error(c, "the environments") != HOTRG_OK) return HOTRG_ECUDA;
  // ---- eigen-decomposition (Sec. 4.2.5), batched over matrices of equal size
  auto eig_batch = [&](const double* Ag, double* Wg, double* Vg, int n, int cnt, int* sweeps_out) -> int {
    const long long nn = (long long)n * n;
    const double* Ainit = Ag;
    if (n >= 32) {
      Phase phw(c, 9);
      // FP32 warm start, FP64 re-orthonormalisation of its vectors (two Newton-Schulz
      // steps Q <- Q (3I - Q^T Q) / 2), W = A Q; the FP64 sweeps then start from (W, Q)
      float* W32 = (float*)c->J32.p;
      float* V32 = W32 + cnt * nn;
      double* G = (double*)c->Gns.p;
      double* Vt = (double*)c->Vtmp.p;
      int ok32;
      {
        Phase ph32(c, 10);
        // at most 15 FP32 sweeps: on 3D chi = 16 (steps 9-28) a cap of 15 against 30 leaves the
        // FP64 sweeps nearly unchanged and saves ~1 ms per step; 10 or 6 cost more FP64 sweeps
        ok32 = launch_jacobi32_block(Ag, W32, V32, n, cnt, 15, (int*)c->counters.p + kCounters32, s) == 0;
        if (!ok32) cudaGetLastError();
      }
      if (ok32) {
        launch_widen_f32(V32, Vg, cnt * nn, s);
        for (int it = 0; it < 2; ++it) {
          launch_gemm_nt_f64_batched(Vg, n, Vg, n, G, n, n, n, n, cnt, nn, nn, nn, s);
          launch_ns_coeff(G, n, cnt, s);
          launch_gemm_nn_f64(G, n, Vg, n, Vt, n, n, n, n, cnt, nn, nn, nn, s);
          cudaMemcpyAsync(Vg, Vt, sizeof(double) * cnt * nn, cudaMemcpyDeviceToDevice, s);
        }
        launch_gemm_nt_f64_batched(Vg, n, Ag, n, Wg, n, n, n, n, cnt, nn, nn, nn, s);
        Ainit = nullptr;
      }
    }
    return launch_jacobi(Wg, Vg, Ainit, n, cnt, 60, (int*)c->counters.p,
                         (unsigned long long*)((int*)c->counters.p + kColmaxOff), sweeps_out,
                         (DevState*)c->state.p, s);
  };
  if (!env_phase) {
    // PH_CONTRACT / PH_FINISH: the isometries were installed by PH_ISO
  } else if (!z2g) {
    for (int g = 0; g < ngrp; ++g) {
      Phase ph(c, 2);
      int cnt = 0;
      long long base = -1;
      for (int j = 1; j < d; ++j)
        if (grp_of[j] == g) {
          cnt += 2;
          if (base < 0 || mat_elem_off[2 * j] < base) base = mat_elem_off[2 * j];
        }
      if (eig_batch((const double*)c->Amat.p + base, (double*)c->W.p + base, (double*)c->V.p + base,
                    grp_n[g], cnt, (int*)c->sweeps.p + grp_first_mat[g]) != 0)
        return launch_failed(c, "Jacobi", grp_n[g], cnt, 0);
    }
  } else {
    // A^(j), A'^(j) are block diagonal in the parity of (hat, check): gather the blocks
    // (both blocks of a leg zero-padded to the larger, so that one launch decomposes
    // them), decompose each size group, scatter W and V back (zeros between parities)
    Phase ph(c, 2);
    const int* zi = (const int*)((const long long*)c->Zg.p + gz_n64);
    long long boff[kMaxD][2][2];
    int bidx[kMaxD][2][2], npad[kMaxD];
    std::vector<int> sizes;
    for (int j = 1; j < d; ++j) {
      npad[j] = std::max(eig_nb[j][0], eig_nb[j][1]);
      if (std::find(sizes.begin(), sizes.end(), npad[j]) == sizes.end()) sizes.push_back(npad[j]);
    }
    long long eoff = 0;
    int nblk = 0;
    std::vector<std::pair<long long, int>> grp_first(sizes.size());   // element offset, block index
    std::vector<int> grp_cnt(sizes.size(), 0);
    for (size_t g = 0; g < sizes.size(); ++g) {
      grp_first[g] = {eoff, nblk};
      for (int j = 1; j < d; ++j)
        for (int k = 0; k < 2; ++k)
          for (int b = 0; b < 2; ++b)
            if (eig_nb[j][b] > 0 && npad[j] == sizes[g]) {
              boff[j][k][b] = eoff;
              bidx[j][k][b] = nblk++;
              eoff += (long long)sizes[g] * sizes[g];
              ++grp_cnt[g];
            }
    }
    CHECK_ALLOC(dev_alloc(c, c->Eb, sizeof(double) * 3 * std::max<long long>(eoff, 1)));
    // the warm start's scratch holds one size group: padded blocks can outgrow the dense
    // matrices (4 npad^2 > 2 n^2 when one parity holds more than 0.707 of a leg's states)
    CHECK_ALLOC(dev_alloc(c, c->J32, sizeof(float) * 2 * std::max<long long>(eoff, 1)));
    CHECK_ALLOC(dev_alloc(c, c->Gns, sizeof(double) * std::max<long long>(eoff, 1)));
    CHECK_ALLOC(dev_alloc(c, c->Vtmp, sizeof(double) * std::max<long long>(eoff, 1)));
    double* Ab = (double*)c->Eb.p;
    double* Wb = Ab + eoff;
    double* Vb = Wb + eoff;
    for (int j = 1; j < d; ++j)
      for (int k = 0; k < 2; ++k)
        for (int b = 0; b < 2; ++b)
          if (eig_nb[j][b] > 0)
            launch_z2_gather_sym((const double*)c->Amat.p + mat_elem_off[2 * j + k], chij[j] * chij[j],
                                 zi + gz_eig[j] + (b == 0 ? 0 : eig_nb[j][0]), eig_nb[j][b], npad[j],
                                 Ab + boff[j][k][b], s);
    int* swb = (int*)c->sweeps.p + 2 * kMaxD;
    for (size_t g = 0; g < sizes.size(); ++g) {
      const long long o = grp_first[g].first;
      if (eig_batch(Ab + o, Wb + o, Vb + o, sizes[g], grp_cnt[g], swb + grp_first[g].second) != 0)
        return launch_failed(c, "Jacobi (Z2 blocks)", sizes[g], grp_cnt[g], 0);
    }
    SweepMerge sm;
    sm.n = 2 * (d - 1);
    for (int j = 1; j < d; ++j) {
      const int n = chij[j] * chij[j];
      const int* eb = zi + gz_eig[j] + n;
      for (int k = 0; k < 2; ++k) {
        const int mat = mat_of_leg[j] + k;
        sm.a[mat] = eig_nb[j][0] > 0 ? bidx[j][k][0] : -1;
        sm.b[mat] = eig_nb[j][1] > 0 ? bidx[j][k][1] : -1;
        const double* w0 = eig_nb[j][0] > 0 ? Wb + boff[j][k][0] : nullptr;
        const double* w1 = eig_nb[j][1] > 0 ? Wb + boff[j][k][1] : nullptr;
        const double* v0 = eig_nb[j][0] > 0 ? Vb + boff[j][k][0] : nullptr;
        const double* v1 = eig_nb[j][1] > 0 ? Vb + boff[j][k][1] : nullptr;
        launch_z2_scatter_eig(w0, w1, npad[j], eb, eb + n, n, (double*)c->W.p + mat_elem_off[2 * j + k], s);
        launch_z2_scatter_eig(v0, v1, npad[j], eb, eb + n, n, (double*)c->V.p + mat_elem_off[2 * j + k], s);
      }
    }
    launch_z2_merge_sweeps(swb, sm, (int*)c->sweeps.p, s);
  }

  if (pending_error(c, "the eigen-solver") != HOTRG_OK) return HOTRG_ECUDA;
  // ---- choice, truncation, gauge (Secs. 4.2.6-4.2.8)
  long long lam_total = 0, u_total = 0;
  long long lam_off[kMaxD], u_off[kMaxD];
  for (int j = 1; j < d; ++j) {
    lam_off[j] = lam_total;
    lam_total += 2LL * chij[j] * chij[j];
    u_off[j] = u_total;
    u_total += (long long)chij[j] * chij[j] * nnew[j];
  }
  CHECK_ALLOC(dev_alloc(c, c->lam, sizeof(double) * lam_total));
  CHECK_ALLOC(dev_alloc(c, c->U64, sizeof(double) * u_total));
  CHECK_ALLOC(dev_alloc(c, c->U32, sizeof(float) * u_total));
  CHECK_ALLOC(dev_alloc(c, c->legres, sizeof(LegResult) * kMaxD));
  long long rank_off[kMaxD], rank_total = 0;
  for (int j = 1; j < d; ++j) {
    rank_off[j] = rank_total;
    rank_total += (long long)chij[j] * chij[j];
  }
  if (tangent) CHECK_ALLOC(dev_alloc(c, c->rank, sizeof(int) * rank_total));
  for (int j = 1; j < d && env_phase; ++j) {
    Phase ph(c, 3);
    int n = chij[j] * chij[j];
    // select_kernel addresses matrices 2*leg_index, 2*leg_index+1 from a base
    launch_select((const double*)c->W.p + mat_elem_off[2 * j], (const double*)c->V.p + mat_elem_off[2 * j],
                  n, 0, nnew[j], (double*)c->lam.p + lam_off[j], (double*)c->U64.p + u_off[j],
                  (float*)c->U32.p + u_off[j], (LegResult*)c->legres.p + j,
                  (int*)c->sweeps.p + mat_of_leg[j], s, tangent ? (int*)c->rank.p + rank_off[j] : nullptr);
  }

  if (pending_error(c, "the selection") != HOTRG_OK) return HOTRG_ECUDA;
  // ---- Z2 blocks at zero field: the parity of each new index is that of the rows
  // its column of U occupies (every nonzero row of a column must agree; a column
  // that mixes parities ends the block treatment for the rest of the run)
  // (parities are tracked while known, and used when the block form is enabled)
  bool z2 = false, track = false;
  std::vector<unsigned char> newpar[kMaxD];
  if (!env_phase) {
    z2 = c->shard_z2 != 0;
    track = c->shard_track != 0;
    for (int j = 1; j < d; ++j) newpar[j] = c->shard_par[j];
  } else if (c->z2_valid) {
    std::vector<double> hu((size_t)u_total);
    if (cudaMemcpyAsync(hu.data(), c->U64.p, sizeof(double) * u_total, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return cuda_status(c) == HOTRG_OK ? (c->poisoned = HOTRG_ECUDA) : HOTRG_ECUDA;
    bool pure = true;
    for (int j = 1; j < d && pure; ++j) {
      const std::vector<unsigned char>& pj = c->par[to[j]];
      const int chj = chij[j], n = chj * chj;
      if ((int)pj.size() != chj) {
        pure = false;
        break;
      }
      newpar[j].assign(nnew[j], 0);
      for (int col = 0; col < nnew[j]; ++col) {
        int seen = -1;
        for (int r = 0; r < n; ++r) {
          if (hu[u_off[j] + (long long)r * nnew[j] + col] == 0.0) continue;
          const int pr = pj[r % chj] ^ pj[r / chj];
          if (seen < 0) seen = pr;
          else if (seen != pr) pure = false;
        }
        newpar[j][col] = (unsigned char)(seen < 0 ? 0 : seen);
      }
    }
    if (pure) {
      track = true;
      z2 = c->z2_enabled != 0 && !tangent;
    } else {
      c->z2_valid = 0;
    }
  }

  if (pending_error(c, "the parity read-back") != HOTRG_OK) return HOTRG_ECUDA;
  if (phase == PH_ISO) {
    // the isometries of this step stay in the context for PH_CONTRACT and PH_FINISH
    c->shard_z2 = z2 ? 1 : 0;
    c->shard_track = track ? 1 : 0;
    for (int j = 1; j < d; ++j) c->shard_par[j] = newpar[j];
    c->shard_axis = axis;
    c->shard_chi = chi;
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_status(c);
    const int r = cuda_status(c);
    if (r == HOTRG_OK) c->shard_ready = 1;
    return r;
  }
  // ---- d/d beta of the chosen environments and of the kept eigenvectors
  // dS = dX X^T + X dX^T (Sec. 3.2), dA = sum dS^ S~ + S^ dS~ (Sec. 4.2.4), and
  // du_k = sum_{l discarded} v_l (v_l . dA u_k) / (lam_k - lam_l) (Sec. 4.2.5)
  if (tangent) {
    Phase ph(c, 1);
    LegResult hres[kMaxD];
    if (cudaMemcpyAsync(hres, c->legres.p, sizeof(LegResult) * kMaxD, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return cuda_status(c) == HOTRG_OK ? (c->poisoned = HOTRG_ECUDA) : HOTRG_ECUDA;
    long long eig_max = 1;
    for (int j = 1; j < d; ++j) eig_max = std::max<long long>(eig_max, (long long)chij[j] * chij[j] * nnew[j]);
    CHECK_ALLOC(dev_alloc(c, c->dXp, sizeof(double) * RR));
    CHECK_ALLOC(dev_alloc(c, c->dS, sizeof(double) * 4 * nlegs * mmax * mmax));
    CHECK_ALLOC(dev_alloc(c, c->dA, sizeof(double) * total_mat_elems));
    CHECK_ALLOC(dev_alloc(c, c->dU64, sizeof(double) * u_total));
    CHECK_ALLOC(dev_alloc(c, c->eG, sizeof(double) * eig_max));
    CHECK_ALLOC(dev_alloc(c, c->eZ, sizeof(double) * eig_max));
    CHECK_ALLOC(dev_alloc(c, c->eZt, sizeof(double) * eig_max));
    long long nmax2 = 1;
    for (int j = 1; j < d; ++j) nmax2 = std::max<long long>(nmax2, (long long)chij[j] * chij[j] * chij[j] * chij[j]);
    if (tan2) {
      CHECK_ALLOC(dev_alloc(c, c->d2Xp, sizeof(double) * RR));
      CHECK_ALLOC(dev_alloc(c, c->d2S, sizeof(double) * 4 * nlegs * mmax * mmax));
      CHECK_ALLOC(dev_alloc(c, c->d2A, sizeof(double) * total_mat_elems));
      CHECK_ALLOC(dev_alloc(c, c->d2U64, sizeof(double) * u_total));
      CHECK_ALLOC(dev_alloc(c, c->eG1, sizeof(double) * nmax2));
      CHECK_ALLOC(dev_alloc(c, c->eW, sizeof(double) * nmax2));
      CHECK_ALLOC(dev_alloc(c, c->eZ2, sizeof(double) * eig_max));
      CHECK_ALLOC(dev_alloc(c, c->eZ2t, sizeof(double) * eig_max));
      CHECK_ALLOC(dev_alloc(c, c->parts2, c->parts.bytes * 2));
    }
    TanState* tst = (TanState*)c->tstate.p;
    for (int j = 1; j < d; ++j) {
      const long long m = (long long)chij[j] * chi_c;
      const long long K = RR / m;
      const int side = hres[j].chose_prime;   // 0: A^(j), 1: A'^(j)
      double* dS0 = (double*)c->dS.p + ((long long)(j - 1) * 4) * mmax * mmax;
      for (int kind = 2 * side; kind < 2 * side + 2; ++kind) {
        long long size[kMaxDims], ist[kMaxDims];
        int pslot[kMaxDims];
        const int nd = gram_dims(j, kind, size, ist, pslot);
        if (z2g) {   // parity blocks, as for the step's own Grams: P_b = dX_b X_b^T
          const long long* zg = (const long long*)c->Zg.p;
          double* X = (double*)c->Xp.p;
          double* dX = (double*)c->dXp.p;
          launch_z2_gather_rc(Tc, zg + gz_roff[j][kind], (int)m, zg + gz_koff[j][kind], K, X, s);
          launch_z2_gather_rc((const double*)c->dT.p, zg + gz_roff[j][kind], (int)m, zg + gz_koff[j][kind], K, dX,
                              s);
          const double* pb[2] = {(const double*)c->parts.p, (const double*)c->parts.p};
          int nsb[2] = {0, 0};
          long long poff = 0;
          for (int b = 0; b < 2; ++b) {
            const long long mb = gz_mb[j][b], Kb = gz_Kb[j][kind][b];
            if (mb == 0 || Kb == 0) continue;
            const long long r0 = b == 0 ? 0 : gz_mb[j][0], q0 = b == 0 ? 0 : gz_Kb[j][kind][0];
            const int nsplit = gram_splits(mb, Kb);
            double* pdst = (double*)c->parts.p + poff;
            nsb[b] = launch_gemm_nt_f64(dX + r0 * K + q0, K, X + r0 * K + q0, K, pdst, mb, mb * mb, (int)mb,
                                        (int)mb, Kb, nsplit, 0, s);
            pb[b] = pdst;
            poff += (long long)nsb[b] * mb * mb;
          }
          const int* zi = (const int*)(zg + gz_n64) + gz_rowmap[j];
          launch_z2_reduce_sum_t(pb[0], nsb[0], (int)gz_mb[j][0], pb[1], nsb[1], (int)gz_mb[j][1], zi, zi + m,
                                 (int)m, dS0 + kind * mmax * mmax, s);
          continue;
        }
        launch_permute(Tc, (double*)c->Xp.p, nd, size, ist, 1.0, s);
        launch_permute((const double*)c->dT.p, (double*)c->dXp.p, nd, size, ist, 1.0, s);
        const int nsplit = gram_splits(m, K);
        const int used = launch_gemm_nt_f64((const double*)c->dXp.p, K, (const double*)c->Xp.p, K,
                                            (double*)c->parts.p, m, m * m, (int)m, (int)m, K, nsplit, 0, s);
        launch_sym_sum((const double*)c->parts.p, used, (int)m, dS0 + kind * mmax * mmax, s);
        if (tan2) {
          // d2S = d2X X^T + X d2X^T + 2 dX dX^T: the partials of d2X X^T and of dX dX^T (each
          // partial of the latter symmetric) summed with their transposes in one pass
          double* d2S0 = (double*)c->d2S.p + ((long long)(j - 1) * 4) * mmax * mmax;
          launch_permute((const double*)c->d2T.p, (double*)c->d2Xp.p, nd, size, ist, 1.0, s);
          double* p2 = (double*)c->parts2.p;
          const int u1 = launch_gemm_nt_f64((const double*)c->d2Xp.p, K, (const double*)c->Xp.p, K, p2, m, m * m,
                                            (int)m, (int)m, K, nsplit, 0, s);
          const int u2 = launch_gemm_nt_f64((const double*)c->dXp.p, K, (const double*)c->dXp.p, K,
                                            p2 + (long long)u1 * m * m, m, m * m, (int)m, (int)m, K, nsplit, 0, s);
          launch_sym_sum(p2, u1 + u2, (int)m, d2S0 + kind * mmax * mmax, s);
        }
      }
      const double* S0 = (const double*)c->S.p + ((long long)(j - 1) * 4) * mmax * mmax;
      const long long k0 = 2 * side;
      double* dAs = (double*)c->dA.p + mat_elem_off[2 * j + side];
      launch_assemble_dot(S0 + k0 * mmax * mmax, dS0 + k0 * mmax * mmax, S0 + (k0 + 1) * mmax * mmax,
                          dS0 + (k0 + 1) * mmax * mmax, chij[j], chi_c, dAs, s);
      const int n = chij[j] * chij[j], nn = nnew[j];
      const double* Vs = (const double*)c->V.p + mat_elem_off[2 * j + side];   // rows: eigenvectors
      double* G = (double*)c->eG.p;
      launch_gemm_nn_f64(dAs, n, (const double*)c->U64.p + u_off[j], nn, G, nn, n, nn, n, 1, 0, 0, 0, s);
      launch_gemm_nn_f64(Vs, n, G, nn, (double*)c->eZ.p, nn, n, nn, n, 1, 0, 0, 0, s);    // v_i . dA u_k
      launch_eig_dscale((const double*)c->eZ.p, (const double*)c->lam.p + lam_off[j] + (long long)side * n,
                        (const int*)c->rank.p + rank_off[j], n, nn, fp64 ? 1e-12 : 1e-8, (double*)c->eZt.p,
                        tst, s);
      launch_gemm_nn_f64((const double*)c->eZt.p, n, Vs, n, G, n, nn, n, n, 1, 0, 0, 0, s);   // dU^T
      launch_transpose(G, nn, n, (double*)c->dU64.p + u_off[j], s);
      if (tan2) {
        // d2A, then d2U = V^T Z2 with Z2 from the projector's second derivative (eig_d2):
        // G1 = V dA V^T over the unsorted eigenvectors, Gs = eZ (v_i . dA u_k), G2s = V d2A U
        const double* d2S0 = (const double*)c->d2S.p + ((long long)(j - 1) * 4) * mmax * mmax;
        double* d2As = (double*)c->d2A.p + mat_elem_off[2 * j + side];
        launch_assemble_ddot(S0 + k0 * mmax * mmax, dS0 + k0 * mmax * mmax, d2S0 + k0 * mmax * mmax,
                             S0 + (k0 + 1) * mmax * mmax, dS0 + (k0 + 1) * mmax * mmax,
                             d2S0 + (k0 + 1) * mmax * mmax, chij[j], chi_c, d2As, s);
        launch_gemm_nn_f64(Vs, n, dAs, n, (double*)c->eW.p, n, n, n, n, 1, 0, 0, 0, s);       // rows dA v_a
        launch_gemm_nt_f64((const double*)c->eW.p, n, Vs, n, (double*)c->eG1.p, n, 0, n, n, n, 1, 0, s);
        launch_gemm_nn_f64(d2As, n, (const double*)c->U64.p + u_off[j], nn, G, nn, n, nn, n, 1, 0, 0, 0, s);
        launch_gemm_nn_f64(Vs, n, G, nn, (double*)c->eZ2.p, nn, n, nn, n, 1, 0, 0, 0, s);    // v_i . d2A u_k
        launch_eig_d2((const double*)c->eG1.p, (const double*)c->eZ.p, (const double*)c->eZ2.p,
                      (const double*)c->lam.p + lam_off[j] + (long long)side * n,
                      (const int*)c->rank.p + rank_off[j], n, nn, 1e-12, (double*)c->eZ2t.p, s);
        launch_gemm_nn_f64((const double*)c->eZ2t.p, n, Vs, n, G, n, nn, n, n, 1, 0, 0, 0, s);   // d2U^T
        launch_transpose(G, nn, n, (double*)c->d2U64.p + u_off[j], s);
      }
    }
    if (!fp64) {
      CHECK_ALLOC(dev_alloc(c, c->dU32, sizeof(float) * u_total));
      launch_narrow_f64((const double*)c->dU64.p, (float*)c->dU32.p, u_total, s);
    }
    if (pending_error(c, "the derivative of the isometries") != HOTRG_OK) return HOTRG_ECUDA;
  }
  // ---- new tensor (Sec. 4.2.9), one c'-slice at a time
  double bn_done = 0.0;
  CHECK_ALLOC(dev_alloc(c, c->T2, sizeof(double) * Rn * Rn));
  double* Tn = (double*)c->T2.p;
  // derivative of the new tensor: the terms through dU^(1) of the last non-prime
  // stage land in dTn2 and are added at the end
  double* dTn = nullptr;
  double* dTn2 = nullptr;
  if (tangent) {
    CHECK_ALLOC(dev_alloc(c, c->dT2, sizeof(double) * Rn * Rn));
    CHECK_ALLOC(dev_alloc(c, c->dTb, sizeof(double) * Rn * Rn));
    dTn = (double*)c->dT2.p;
    dTn2 = (double*)c->dTb.p;
  }
  // second order: the three terms of the last non-prime stage land in d2Tn, d2Tn2 (the
  // cross term, doubled at the end) and d2Tn3
  double *d2Tn = nullptr, *d2Tn2 = nullptr, *d2Tn3 = nullptr;
  if (tan2) {
    CHECK_ALLOC(dev_alloc(c, c->d2T2, sizeof(double) * Rn * Rn));
    CHECK_ALLOC(dev_alloc(c, c->d2Tb, sizeof(double) * Rn * Rn));
    CHECK_ALLOC(dev_alloc(c, c->d2Tc, sizeof(double) * Rn * Rn));
    d2Tn = (double*)c->d2T2.p;
    d2Tn2 = (double*)c->d2Tb.p;
    d2Tn3 = (double*)c->d2Tc.p;
  }
  // the c'-slices this call contracts (all of them but in PH_CONTRACT)
  const int sl_lo = phase == PH_CONTRACT ? sh.c_lo : 0;
  const int sl_hi = phase == PH_CONTRACT ? sh.c_hi : chi_c;
  const long long slice_elems = Rn * Pn;   // one c'-slice of T': Rn rows x Pn columns (n')
  if (phase == PH_CONTRACT) {
    if (sh.n_out) *sh.n_out = (long long)std::max(0, sl_hi - sl_lo) * slice_elems;
    if (sl_lo < 0 || sl_hi > chi_c || sl_lo >= sl_hi || !sh.out ||
        sh.cap < (long long)(sl_hi - sl_lo) * slice_elems)
      return HOTRG_EINVAL;
  }
  if (phase == PH_FINISH && (!sh.in || sh.cap != (long long)chi_c * slice_elems)) return HOTRG_EINVAL;
  if (phase == PH_FULL || phase == PH_CONTRACT) {
  const long long Ns = Pn * P;            // columns of the bottleneck per slice: (n', n~)
  const int npieces = split_pieces(c->precision);
  const int pfmt = split_format(c->precision);
  const long long pbytes = piece_bytes(pfmt);
  const long long Kpad = fp64 ? R : (R + 63) / 64 * 64;
  // chain intermediates
  long long chain_max = 1;
  {
    long long acc = 1;
    for (int j = 1; j < d - 1; ++j) {
      acc *= nnew[j];
      chain_max = std::max(chain_max, acc * chi_c * P * P);
    }
    for (int j = d - 1; j > 1; --j) {
      long long hat = 1;
      for (int k = 1; k < j; ++k) hat *= chij[k];
      long long nn_tail = 1;
      for (int k = j; k < d; ++k) nn_tail *= nnew[k];
      chain_max = std::max(chain_max, (long long)chi_c * hat * Pn * hat * nn_tail);
    }
  }
  size_t elt = (fp64 || c->f64_chains) ? sizeof(double) : sizeof(float);
  // Sub-slices of n'_1 keep the per-slice operands within a device-memory budget:
  // everything below except the split T scales with the number of n'_1 values.
  const int nnew1 = nnew[1];
  int n1_chunk = nnew1;
  {
    // the Z2 blocks of B and C hold about half of B and C again; the derivative
    // adds two more of B and C (and FP64 staging of dB in the split form) and three
    // more chain buffers
    const double per_unit =
        (z2 ? 1.6 : 1.0) * (tangent ? (fp64 ? (tan2 ? 4.0 : 3.0) : 4.0) : 1.0) * (double)(Ns / nnew1) *
            ((fp64 ? 8.0 * R : (double)pbytes * npieces * Kpad) + (fp64 ? 8.0 : 4.0) * R) +
        (tan2 ? 7.0 : (tangent ? 5.0 : 2.0)) * (double)elt * (double)chain_max / nnew1;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    double budget = std::min(0.6 * (double)free_b + (double)(c->Bp.bytes + c->Cb.bytes + c->chA.bytes +
                                                             c->chB.bytes + c->Zb.bytes + c->Zc.bytes),
                             c->slice_budget_bytes);
    n1_chunk = (int)std::max(1.0, std::min((double)nnew1, std::floor(budget / per_unit)));
  }
  const long long Nsub = (long long)n1_chunk * (Ns / nnew1);
  const long long chain_sub = (chain_max / nnew1) * n1_chunk;
  CHECK_ALLOC(dev_alloc(c, c->chA, elt * chain_sub));
  CHECK_ALLOC(dev_alloc(c, c->chB, elt * chain_sub));
  if (tangent) {
    CHECK_ALLOC(dev_alloc(c, c->dchA, elt * chain_sub));
    CHECK_ALLOC(dev_alloc(c, c->dchB, elt * chain_sub));
    CHECK_ALLOC(dev_alloc(c, c->dchT, elt * chain_sub));
  }
  if (tan2) {
    CHECK_ALLOC(dev_alloc(c, c->d2chA, elt * chain_sub));
    CHECK_ALLOC(dev_alloc(c, c->d2chB, elt * chain_sub));
  }
  // Z2 index maps.  Rows of T and the contracted index (rho, n^') run over the same
  // slots with the same parities, so one list per parity b serves as the row map
  // (first R_b entries) and, padded with -1 to Kp_b, as the K map of block b.
  long long Rb[2] = {0, 0}, Kpb[2] = {0, 0}, maxL = 0;
  long long moff_rowblk = 0, moff_rowpos = 0, moff_kcat = 0, moff_k[2] = {0, 0};
  struct Z2Chunk {
    long long off_blk, off_pos, off_list[2], L[2];
  };
  std::vector<Z2Chunk> zch;
  if (z2) {
    std::vector<int> hmap;
    auto push = [&](const std::vector<int>& v) {
      long long off = (long long)hmap.size();
      hmap.insert(hmap.end(), v.begin(), v.end());
      while (hmap.size() % 4) hmap.push_back(0);
      return off;
    };
    // Each parity's list runs over the last slot's index slowest (any order serves, as
    // long as the A blocks, the B blocks and the C rows share it): in this order the
    // consecutive list positions that the lanes of a warp take in the last prime stage
    // share the hat index of the last leg, so they read one isometry row
    std::vector<int> rowblk(R), rowpos(R), kmap[2];
    const int chi_last = c->chis[to[d - 1]];
    const long long rest = R / chi_last;
    for (long long o = 0; o < R; ++o) {
      const long long r = (o % rest) * chi_last + o / rest;
      long long idx = r;
      int p_ = 0;
      for (int k = d - 1; k >= 0; --k) {
        const int sz = c->chis[to[k]];
        p_ ^= c->par[to[k]][idx % sz];
        idx /= sz;
      }
      rowblk[r] = p_;
      rowpos[r] = (int)kmap[p_].size();
      kmap[p_].push_back((int)r);
    }
    for (int b = 0; b < 2; ++b) Rb[b] = (long long)kmap[b].size();
    {
      // the contracted index (rho, n^') runs over the same slots as the rows: both K
      // lists back to back (parity 0, then parity 1), without padding
      std::vector<int> kcat(kmap[0].begin(), kmap[0].end());
      kcat.insert(kcat.end(), kmap[1].begin(), kmap[1].end());
      moff_kcat = push(kcat);
    }
    for (int b = 0; b < 2; ++b) {
      Kpb[b] = fp64 ? Rb[b] : (Rb[b] + 63) / 64 * 64;
      kmap[b].resize(Kpb[b], -1);
    }
    moff_rowblk = push(rowblk);
    moff_rowpos = push(rowpos);
    for (int b = 0; b < 2; ++b) moff_k[b] = push(kmap[b]);
    // parity of a bottleneck column (n', n~): new legs from U, old legs as before
    std::vector<unsigned char> pnp((size_t)Pn), ptl((size_t)P);
    for (long long x = 0; x < Pn; ++x) {
      long long idx = x;
      int p_ = 0;
      for (int k = d - 1; k >= 1; --k) {
        p_ ^= newpar[k][idx % nnew[k]];
        idx /= nnew[k];
      }
      pnp[x] = (unsigned char)p_;
    }
    for (long long x = 0; x < P; ++x) {
      long long idx = x;
      int p_ = 0;
      for (int k = d - 1; k >= 1; --k) {
        p_ ^= c->par[to[k]][idx % chij[k]];
        idx /= chij[k];
      }
      ptl[x] = (unsigned char)p_;
    }
    const long long per_n1 = Ns / nnew1;
    for (int n1lo = 0; n1lo < nnew1; n1lo += n1_chunk) {
      const long long Nc = (long long)std::min(n1_chunk, nnew1 - n1lo) * per_n1;
      const long long base = (long long)n1lo * per_n1;
      std::vector<int> colblk(Nc), colpos(Nc), lst[2];
      for (long long n = 0; n < Nc; ++n) {
        const long long g = base + n;
        const int p_ = pnp[g / P] ^ ptl[g % P];
        colblk[n] = p_;
        colpos[n] = (int)lst[p_].size();
        lst[p_].push_back((int)n);
      }
      Z2Chunk ch;
      ch.off_blk = push(colblk);
      ch.off_pos = push(colpos);
      for (int b = 0; b < 2; ++b) {
        ch.off_list[b] = push(lst[b]);
        ch.L[b] = (long long)lst[b].size();
        maxL = std::max(maxL, ch.L[b]);
      }
      zch.push_back(ch);
    }
    CHECK_ALLOC(dev_alloc(c, c->Zmap, sizeof(int) * hmap.size()));
    if (cudaMemcpyAsync(c->Zmap.p, hmap.data(), sizeof(int) * hmap.size(), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return cuda_status(c) == HOTRG_OK ? (c->poisoned = HOTRG_ECUDA) : HOTRG_ECUDA;
  }
  const int* zmap = (const int*)c->Zmap.p;
  // split form with Z2 blocks: the last prime stage writes the B blocks directly (no
  // dense B, no gather) and the first non-prime stage reads the product's blocks
  // directly (no dense C)
  const bool zfold = z2 && !fp64 && !c->f64_chains;
  const long long ldz = (maxL + 3) / 4 * 4;   // row pitch of the C blocks
  if (fp64) {
    CHECK_ALLOC(dev_alloc(c, c->Bp, sizeof(double) * Nsub * R));
    CHECK_ALLOC(dev_alloc(c, c->Cb, sizeof(double) * R * Nsub));
    if (tangent) {
      CHECK_ALLOC(dev_alloc(c, c->dBp, sizeof(double) * Nsub * R));
      CHECK_ALLOC(dev_alloc(c, c->tBp, sizeof(double) * Nsub * R));
      CHECK_ALLOC(dev_alloc(c, c->dCb, sizeof(double) * R * Nsub));
      CHECK_ALLOC(dev_alloc(c, c->tCb, sizeof(double) * R * Nsub));
    }
    if (tan2) {
      CHECK_ALLOC(dev_alloc(c, c->d2Bp, sizeof(double) * Nsub * R));
      CHECK_ALLOC(dev_alloc(c, c->d2Cb, sizeof(double) * R * Nsub));
    }
    if (z2) {
      CHECK_ALLOC(dev_alloc(c, c->Za, sizeof(double) * (Rb[0] * Kpb[0] + Rb[1] * Kpb[1])));
      CHECK_ALLOC(dev_alloc(c, c->Zb, sizeof(double) * maxL * (Kpb[0] + Kpb[1])));
      CHECK_ALLOC(dev_alloc(c, c->Zc, sizeof(double) * R * ldz));
      double* za = (double*)c->Za.p;
      launch_z2_gather_f64(Tc, R, zmap + moff_k[0], (int)Rb[0], zmap + moff_k[0], (int)Kpb[0], za, s);
      launch_z2_gather_f64(Tc, R, zmap + moff_k[1], (int)Rb[1], zmap + moff_k[1], (int)Kpb[1],
                           za + Rb[0] * Kpb[0], s);
    }
  } else {
    if (!zfold) {   // with the Z2 blocks the last prime stage writes the B blocks directly
      CHECK_ALLOC(dev_alloc(c, c->Bp, pbytes * npieces * Nsub * Kpad));
      if (Kpad != R) cudaMemsetAsync(c->Bp.p, 0, pbytes * npieces * Nsub * Kpad, s);
      CHECK_ALLOC(dev_alloc(c, c->Cb, sizeof(float) * R * Nsub));
    }
    if (tangent) {
      CHECK_ALLOC(dev_alloc(c, c->dBp, pbytes * npieces * Nsub * Kpad));
      if (Kpad != R) cudaMemsetAsync(c->dBp.p, 0, pbytes * npieces * Nsub * Kpad, s);
      CHECK_ALLOC(dev_alloc(c, c->dB64, sizeof(double) * Nsub * R));
      CHECK_ALLOC(dev_alloc(c, c->tBp, sizeof(double) * Nsub * R));
      CHECK_ALLOC(dev_alloc(c, c->dCb, sizeof(float) * R * Nsub));
      CHECK_ALLOC(dev_alloc(c, c->tCb, sizeof(float) * R * Nsub));
    }
    Phase ph(c, 4);
    if (z2) {
      CHECK_ALLOC(dev_alloc(c, c->Za, pbytes * npieces * (Rb[0] * Kpb[0] + Rb[1] * Kpb[1])));
      CHECK_ALLOC(dev_alloc(c, c->Zb, pbytes * npieces * maxL * (Kpb[0] + Kpb[1])));
      CHECK_ALLOC(dev_alloc(c, c->Zc, sizeof(float) * R * ldz));
      char* za = (char*)c->Za.p;
      launch_z2_gather_split(Tc, R, zmap + moff_k[0], (int)Rb[0], zmap + moff_k[0], (int)Kpb[0], za,
                             Rb[0] * Kpb[0], npieces, pfmt, s);
      launch_z2_gather_split(Tc, R, zmap + moff_k[1], (int)Rb[1], zmap + moff_k[1], (int)Kpb[1],
                             za + pbytes * npieces * Rb[0] * Kpb[0], Rb[1] * Kpb[1], npieces, pfmt, s);
    } else {
      CHECK_ALLOC(dev_alloc(c, c->Ap, pbytes * npieces * R * Kpad));
      if (Kpad != R) cudaMemsetAsync(c->Ap.p, 0, pbytes * npieces * R * Kpad, s);
      launch_split(Tc, R, R, R, c->Ap.p, Kpad, R * Kpad, npieces, pfmt, s);
      if (tangent) {
        CHECK_ALLOC(dev_alloc(c, c->dAp, pbytes * npieces * R * Kpad));
        if (Kpad != R) cudaMemsetAsync(c->dAp.p, 0, pbytes * npieces * R * Kpad, s);
        launch_split((const double*)c->dT.p, R, R, R, c->dAp.p, Kpad, R * Kpad, npieces, pfmt, s);
      }
    }
  }
  auto view_elems = [](const View& v) {
    long long n_ = 1;
    for (auto& x : v) n_ *= x.size;
    return n_;
  };

  // products of trailing bond sizes
  auto prod_after = [&](const int* arr, int k) {
    long long p_ = 1;
    for (int l = k + 1; l < d; ++l) p_ *= arr[l];
    return p_;
  };
  int terms_a[6], terms_b[6];
  const int nterms = split_terms(npieces, terms_a, terms_b);

  const void* cblk_cur[2] = {nullptr, nullptr};   // this sub-slice's C blocks (Z2)
  for (int sl = sl_lo; sl < sl_hi; ++sl)
  for (int n1lo = 0; n1lo < nnew1; n1lo += n1_chunk) {
    const int n1cnt = std::min(n1_chunk, nnew1 - n1lo);
    const long long Nc = (long long)n1cnt * (Ns / nnew1);   // bottleneck columns of this sub-slice
    int nsz[kMaxD];                                          // n' sizes of this sub-slice
    for (int k = 1; k < d; ++k) nsz[k] = k == 1 ? n1cnt : nnew[k];
    // -- prime-side chain, Eqs. (TU1)-(TUNCD), on the c'-fixed tensor T[(rho, n~), (sl, n~')]
    View in;
    in.push_back({I_RHO, chi_c, rs[0]});
    for (int k = 1; k < d; ++k) in.push_back({I_NC + k, chij[k], rs[k]});
    for (int k = 1; k < d; ++k) in.push_back({I_NCP + k, chij[k], cs[k]});
    const void* src = Tc + (long long)sl * cs[0];
    const void* dsrc = tangent ? (const double*)c->dT.p + (long long)sl * cs[0] : nullptr;
    const void* d2src = tan2 ? (const double*)c->d2T.p + (long long)sl * cs[0] : nullptr;
    int src_f64 = 1;
    for (int j = 1; j < d; ++j) {
      Phase ph(c, 5);
      View out;
      bool last = (j == d - 1);
      if (!last) {
        std::vector<std::pair<int, long long>> names;
        for (int k = 1; k <= j; ++k) names.push_back({I_NP + k, nsz[k]});
        names.push_back({I_RHO, chi_c});
        for (int k = 1; k < d; ++k) names.push_back({I_NC + k, chij[k]});
        for (int k = j + 1; k < d; ++k) names.push_back({I_NCP + k, chij[k]});
        for (int k = 1; k <= j; ++k) names.push_back({I_NHP + k, chij[k]});
        out = contiguous(names);
      } else {
        long long K_ = Kpad;
        for (int k = 1; k < d; ++k) out.push_back({I_NP + k, nsz[k], prod_after(nnew, k) * P * K_});
        for (int k = 1; k < d; ++k) out.push_back({I_NC + k, chij[k], prod_after(chij, k) * K_});
        out.push_back({I_RHO, chi_c, P});
        for (int k = 1; k < d; ++k) out.push_back({I_NHP + k, chij[k], prod_after(chij, k)});
      }
      ChainDesc cd;
      if (!make_stage(cd, in, out, I_NHP + j, I_NCP + j, I_NP + j, chij[j], nsz[j])) {
        c->poisoned = HOTRG_EINVAL;
        return HOTRG_EINVAL;
      }
      // columns n1lo .. n1lo + n1cnt - 1 of U~^(1) give this sub-slice's n'_1
      cd.ldu = nnew[j];
      const long long ucol = j == 1 ? n1lo : 0;
      void* dst = last ? c->Bp.p : ((j & 1) ? c->chA.p : c->chB.p);
      if (fp64) {
        launch_chain_f64(cd, (const double*)src, (const double*)c->U64.p + u_off[j] + ucol, (double*)dst, s);
        if (tangent) {   // dX_j = stage(dX_{j-1}, U) + stage(X_{j-1}, dU)
          double* ddst = last ? (double*)c->dBp.p : (double*)((j & 1) ? c->dchA.p : c->dchB.p);
          double* tdst = last ? (double*)c->tBp.p : (double*)c->dchT.p;
          launch_chain_f64(cd, (const double*)dsrc, (const double*)c->U64.p + u_off[j] + ucol, ddst, s);
          launch_chain_f64(cd, (const double*)src, (const double*)c->dU64.p + u_off[j] + ucol, tdst, s);
          launch_axpby(1.0, tdst, 1.0, ddst, view_elems(out), s);
          if (tan2) {   // d2X_j = stage(d2X_{j-1}, U) + 2 stage(dX_{j-1}, dU) + stage(X_{j-1}, d2U)
            double* d2dst = last ? (double*)c->d2Bp.p : (double*)((j & 1) ? c->d2chA.p : c->d2chB.p);
            launch_chain_f64(cd, (const double*)d2src, (const double*)c->U64.p + u_off[j] + ucol, d2dst, s);
            launch_chain_f64(cd, (const double*)dsrc, (const double*)c->dU64.p + u_off[j] + ucol, tdst, s);
            launch_axpby(2.0, tdst, 1.0, d2dst, view_elems(out), s);
            launch_chain_f64(cd, (const double*)src, (const double*)c->d2U64.p + u_off[j] + ucol, tdst, s);
            launch_axpby(1.0, tdst, 1.0, d2dst, view_elems(out), s);
            d2src = d2dst;
          }
          dsrc = ddst;
        }
      } else if (c->f64_chains && !tangent) {
        cd.npieces = npieces;
        cd.pfmt = pfmt;
        cd.piece_stride = Nc * Kpad;
        launch_chain_f64acc(cd, src, src_f64, (const double*)c->U64.p + u_off[j] + ucol, dst,
                            last ? OUT_BF16_SPLIT : OUT_F64, s);
      } else if (last && zfold) {
        // straight into the Z2 blocks of B: the outputs whose column parity matches
        // the parity of their k, at the positions the bottleneck's blocks use
        cd.npieces = npieces;
        cd.pfmt = pfmt;
        const Z2Chunk& ch = zch[n1lo / n1_chunk];
        const int q = c->par[to[0]][sl];
        Z2Out zo;
        zo.kcat = zmap + moff_kcat;
        zo.R = (unsigned)R;
        zo.rb0 = (unsigned)Rb[0];
        zo.cblk = zmap + ch.off_blk;
        zo.cpos = zmap + ch.off_pos;
        zo.q = q;
        zo.kpad = Kpad;
        zo.nrow_step = cd.n_out_stride / Kpad;
        for (int b = 0; b < 2; ++b) {
          const long long Nb = ch.L[b ^ q];
          char* zb = (char*)c->Zb.p + pbytes * npieces * (b == 0 ? 0 : maxL * Kpb[0]);
          zo.blk[b] = zb;
          zo.ld[b] = Kpb[b];
          zo.pstride[b] = Nb * Kpb[b];
          // the K padding of every row (of every piece) reads as zero
          if (Kpb[b] > Rb[b] && Nb > 0 &&
              cudaMemset2DAsync(zb + pbytes * Rb[b], pbytes * Kpb[b], 0, pbytes * (Kpb[b] - Rb[b]),
                                (size_t)npieces * Nb, s) != cudaSuccess)
            return cuda_status(c) == HOTRG_OK ? (c->poisoned = HOTRG_ECUDA) : HOTRG_ECUDA;
        }
        {
          // the leading free dims of the stage must be exactly the k dims (R values),
          // the others rows of the dense view (strides multiples of Kpad)
          long long kprod = 1;
          int q0 = 0;
          while (q0 < cd.ndim && cd.out_stride[q0] < Kpad) kprod *= cd.size[q0++];
          bool okz = kprod == R && cd.n_out_stride % Kpad == 0;
          for (int q1 = q0; q1 < cd.ndim; ++q1) okz = okz && cd.out_stride[q1] % Kpad == 0;
          for (int q1 = 0; q1 + 1 < cd.ndim; ++q1) okz = okz && cd.out_stride[q1] <= cd.out_stride[q1 + 1];
          if (!okz) {
            c->poisoned = HOTRG_EINVAL;
            return HOTRG_EINVAL;
          }
          // the output row of a thread: sum of its row-dim indices times their strides / Kpad
          for (int q1 = 0; q1 < kMaxDims; ++q1) zo.rstride[q1] = q1 >= q0 && q1 < cd.ndim ? cd.out_stride[q1] / Kpad : 0;
          // t / R by multiply-shift, as for the dims (make_stage)
          int l = 0;
          while ((1ULL << l) < (unsigned long long)R) ++l;
          zo.r_shift = l;
          zo.r_magic = (unsigned)((((1ULL << l) - (unsigned long long)R) << 32) / (unsigned long long)R + 1);
        }
        tuned_chain(c, cd, 1, [&] { launch_chain_f32_z2out(cd, src, src_f64, (const float*)c->U32.p + u_off[j] + ucol, zo, s); });
      } else {
        cd.npieces = npieces;
        cd.pfmt = pfmt;
        cd.piece_stride = Nc * Kpad;
        tuned_chain(c, cd, last ? 3 : 4, [&] {
          launch_chain_f32(cd, src, src_f64, (const float*)c->U32.p + u_off[j] + ucol, dst,
                           last ? OUT_BF16_SPLIT : OUT_F32, s);
        });
        if (tangent) {   // the same in FP32; the last stage sums in FP64 (row pitch R), then splits
          ChainDesc cdt = cd;
          if (last) {
            View outT;
            for (int k = 1; k < d; ++k) outT.push_back({I_NP + k, nsz[k], prod_after(nnew, k) * P * R});
            for (int k = 1; k < d; ++k) outT.push_back({I_NC + k, chij[k], prod_after(chij, k) * R});
            outT.push_back({I_RHO, chi_c, P});
            for (int k = 1; k < d; ++k) outT.push_back({I_NHP + k, chij[k], prod_after(chij, k)});
            if (!make_stage(cdt, in, outT, I_NHP + j, I_NCP + j, I_NP + j, chij[j], nsz[j])) {
              c->poisoned = HOTRG_EINVAL;
              return HOTRG_EINVAL;
            }
            cdt.ldu = nnew[j];
          }
          void* ddst = last ? c->dB64.p : ((j & 1) ? c->dchA.p : c->dchB.p);
          void* tdst = last ? c->tBp.p : c->dchT.p;
          const int mode = last ? OUT_F64 : OUT_F32;
          launch_chain_f32(cdt, dsrc, src_f64, (const float*)c->U32.p + u_off[j] + ucol, ddst, mode, s);
          launch_chain_f32(cdt, src, src_f64, (const float*)c->dU32.p + u_off[j] + ucol, tdst, mode, s);
          if (last) {   // dB = both terms, summed in FP64 as they are split
            launch_split((const double*)ddst, Nc, R, R, c->dBp.p, Kpad, Nc * Kpad, npieces, pfmt, s,
                         (const double*)tdst);
          } else {
            launch_add_f32((const float*)tdst, (float*)ddst, view_elems(out), s);
          }
          dsrc = ddst;
        }
      }
      src = dst;
      src_f64 = (fp64 || (c->f64_chains && !tangent)) ? 1 : 0;
      in = out;
    }
    if (pending_error(c, "the prime chain") != HOTRG_OK) return HOTRG_ECUDA;
    // -- bottleneck, Eq. (BottleneckPart): C[(c, n^)][(n', n~)] = T . B^T
    if (z2) {
      // blocks b = 0, 1: rows and K of parity b, columns of parity b ^ q
      const int q = c->par[to[0]][sl];
      const Z2Chunk& ch = zch[n1lo / n1_chunk];
      const void* cblk[2] = {nullptr, nullptr};
      long long ldb_[2] = {1, 1};
      for (int b = 0; b < 2; ++b) {
        const long long Nb = ch.L[b ^ q];
        if (Rb[b] == 0 || Nb == 0) continue;
        const int* nmap = zmap + ch.off_list[b ^ q];
        const int* kmap = zmap + moff_k[b];
        const long long a_off = b == 0 ? 0 : Rb[0] * Kpb[0];
        const long long b_off = b == 0 ? 0 : maxL * Kpb[0];
        const long long c_off = b == 0 ? 0 : Rb[0] * ldz;
        if (fp64) {
          double* zb = (double*)c->Zb.p + b_off;
          double* zc = (double*)c->Zc.p + c_off;
          {
            Phase pg(c, 11);
            launch_z2_gather_f64((const double*)c->Bp.p, R, nmap, (int)Nb, kmap, (int)Kpb[b], zb, s);
          }
          Phase ph(c, 6);
          launch_gemm_nt_f64((const double*)c->Za.p + a_off, Kpb[b], zb, Kpb[b], zc, ldz, 0, (int)Rb[b],
                             (int)Nb, Kpb[b], 1, 0, s);
          cblk[b] = zc;
        } else {
          char* zb = (char*)c->Zb.p + pbytes * npieces * b_off;
          float* zc = (float*)c->Zc.p + c_off;
          if (!zfold) {   // else the last prime stage wrote the block
            Phase pg(c, 11);
            launch_z2_gather_pieces(c->Bp.p, Kpad, Nc * Kpad, nmap, (int)Nb, kmap, (int)Kpb[b], zb,
                                    Nb * Kpb[b], npieces, pfmt, s);
          }
          Phase ph(c, 6);
          if (launch_tc_gemm((const char*)c->Za.p + pbytes * npieces * a_off, (int)Rb[b], zb, (int)Nb,
                             (int)Kpb[b], npieces, nterms, terms_a, terms_b, zc, ldz,
                             &((DevState*)c->state.p)->status, s, nullptr, pfmt) != 0)
            return launch_failed(c, "tensor-core GEMM (Z2 block)", Rb[b], Nb, Kpb[b]);
          cblk[b] = zc;
        }
        ldb_[b] = ldz;
        bn_done += 2.0 * (double)Rb[b] * (double)Nb * (double)Rb[b];
      }
      for (int b = 0; b < 2; ++b) cblk_cur[b] = cblk[b];
      if (!zfold) {
        Phase pg(c, 11);
        if (fp64)
          launch_z2_scatter_f64((const double*)cblk[0], ldb_[0], (const double*)cblk[1], ldb_[1],
                                zmap + moff_rowblk, zmap + moff_rowpos, zmap + ch.off_blk,
                                zmap + ch.off_pos, q, (int)R, (int)Nc, (double*)c->Cb.p, s);
        else
          launch_z2_scatter_f32((const float*)cblk[0], ldb_[0], (const float*)cblk[1], ldb_[1],
                                zmap + moff_rowblk, zmap + moff_rowpos, zmap + ch.off_blk,
                                zmap + ch.off_pos, q, (int)R, (int)Nc, (float*)c->Cb.p, s);
      }
    } else {
    bn_done += 2.0 * (double)R * (double)Nc * (double)R;
    Phase ph(c, 6);
    if (fp64) {
      launch_gemm_nt_f64(Tc, R, (const double*)c->Bp.p, R, (double*)c->Cb.p, Nc, 0, (int)R, (int)Nc,
                         R, 1, 0, s);
      if (tangent) {   // dC = T^ . dB^T + dT^ . B^T
        launch_gemm_nt_f64(Tc, R, (const double*)c->dBp.p, R, (double*)c->dCb.p, Nc, 0, (int)R, (int)Nc, R, 1,
                           0, s);
        launch_gemm_nt_f64((const double*)c->dT.p, R, (const double*)c->Bp.p, R, (double*)c->tCb.p, Nc, 0,
                           (int)R, (int)Nc, R, 1, 0, s);
        launch_axpby(1.0, (const double*)c->tCb.p, 1.0, (double*)c->dCb.p, R * Nc, s);
      }
      if (tan2) {      // d2C = T^ . d2B^T + 2 dT^ . dB^T + d2T^ . B^T
        launch_gemm_nt_f64(Tc, R, (const double*)c->d2Bp.p, R, (double*)c->d2Cb.p, Nc, 0, (int)R, (int)Nc, R, 1,
                           0, s);
        launch_gemm_nt_f64((const double*)c->dT.p, R, (const double*)c->dBp.p, R, (double*)c->tCb.p, Nc, 0,
                           (int)R, (int)Nc, R, 1, 0, s);
        launch_axpby(2.0, (const double*)c->tCb.p, 1.0, (double*)c->d2Cb.p, R * Nc, s);
        launch_gemm_nt_f64((const double*)c->d2T.p, R, (const double*)c->Bp.p, R, (double*)c->tCb.p, Nc, 0,
                           (int)R, (int)Nc, R, 1, 0, s);
        launch_axpby(1.0, (const double*)c->tCb.p, 1.0, (double*)c->d2Cb.p, R * Nc, s);
      }
    } else {
      if (launch_tc_gemm(c->Ap.p, (int)R, c->Bp.p, (int)Nc, (int)Kpad, npieces, nterms, terms_a, terms_b,
                         (float*)c->Cb.p, Nc, &((DevState*)c->state.p)->status, s, nullptr, pfmt) != 0)
        return launch_failed(c, "tensor-core GEMM", R, Nc, Kpad);
      if (tangent) {   // dC = T^ . dB^T + dT^ . B^T
        if (launch_tc_gemm(c->Ap.p, (int)R, c->dBp.p, (int)Nc, (int)Kpad, npieces, nterms, terms_a, terms_b,
                           (float*)c->dCb.p, Nc, &((DevState*)c->state.p)->status, s, nullptr, pfmt) != 0 ||
            launch_tc_gemm(c->dAp.p, (int)R, c->Bp.p, (int)Nc, (int)Kpad, npieces, nterms, terms_a, terms_b,
                           (float*)c->tCb.p, Nc, &((DevState*)c->state.p)->status, s, nullptr, pfmt) != 0)
          return launch_failed(c, "tensor-core GEMM (derivative)", R, Nc, Kpad);
        launch_add_f32((const float*)c->tCb.p, (float*)c->dCb.p, R * Nc, s);
      }
    }
    }
    if (pending_error(c, "the bottleneck") != HOTRG_OK) return HOTRG_ECUDA;
    // -- non-prime chain, Eqs. (AfterBNNCD)-(AfterBN1), Eq. (Elements_NewTensor)
    View cin;
    // folded Z2 blocks: packed strides (row of C) << 32 | (column of C)
    const long long rsh = zfold ? (1LL << 32) : Nc;
    cin.push_back({I_C, chi_c, P * rsh});
    for (int k = 1; k < d; ++k) cin.push_back({I_NH + k, chij[k], prod_after(chij, k) * rsh});
    for (int k = 1; k < d; ++k) cin.push_back({I_NP + k, nsz[k], prod_after(nnew, k) * P});
    for (int k = 1; k < d; ++k) cin.push_back({I_NC + k, chij[k], prod_after(chij, k)});
    const void* csrc = c->Cb.p;
    const void* dcsrc = tangent ? c->dCb.p : nullptr;
    const void* d2csrc = tan2 ? c->d2Cb.p : nullptr;
    for (int j = d - 1; j >= 1; --j) {
      Phase ph(c, 7);
      View out;
      bool last = (j == 1);
      if (!last) {
        std::vector<std::pair<int, long long>> names;
        names.push_back({I_C, chi_c});
        for (int k = 1; k < j; ++k) names.push_back({I_NH + k, chij[k]});
        for (int k = 1; k < d; ++k) names.push_back({I_NP + k, nsz[k]});
        for (int k = 1; k < j; ++k) names.push_back({I_NC + k, chij[k]});
        for (int k = j; k < d; ++k) names.push_back({I_N + k, nnew[k]});
        out = contiguous(names);
      } else {
        out.push_back({I_C, chi_c, Pn * Rn});
        for (int k = 1; k < d; ++k) out.push_back({I_N + k, nnew[k], prod_after(nnew, k) * Rn});
        for (int k = 1; k < d; ++k) out.push_back({I_NP + k, nsz[k], prod_after(nnew, k)});
      }
      ChainDesc cd;
      if (!make_stage(cd, cin, out, I_NH + j, I_NC + j, I_N + j, chij[j], nnew[j])) {
        c->poisoned = HOTRG_EINVAL;
        return HOTRG_EINVAL;
      }
      void* dst = last ? (void*)(Tn + (long long)sl * Pn + (long long)n1lo * prod_after(nnew, 1))
                       : ((j & 1) ? c->chA.p : c->chB.p);
      if (fp64) {
        launch_chain_f64(cd, (const double*)csrc, (const double*)c->U64.p + u_off[j], (double*)dst, s);
        if (tangent) {   // dY_j = stage(dY_{j+1}, U) + stage(Y_{j+1}, dU)
          const long long slab = (long long)sl * Pn + (long long)n1lo * prod_after(nnew, 1);
          double* ddst = last ? dTn + slab : (double*)((j & 1) ? c->dchA.p : c->dchB.p);
          double* tdst = last ? dTn2 + slab : (double*)c->dchT.p;
          launch_chain_f64(cd, (const double*)dcsrc, (const double*)c->U64.p + u_off[j], ddst, s);
          launch_chain_f64(cd, (const double*)csrc, (const double*)c->dU64.p + u_off[j], tdst, s);
          if (!last) launch_axpby(1.0, tdst, 1.0, ddst, view_elems(out), s);
          if (tan2) {   // d2Y_j = stage(d2Y_{j+1}, U) + 2 stage(dY_{j+1}, dU) + stage(Y_{j+1}, d2U)
            double* d2dst = last ? d2Tn + slab : (double*)((j & 1) ? c->d2chA.p : c->d2chB.p);
            launch_chain_f64(cd, (const double*)d2csrc, (const double*)c->U64.p + u_off[j], d2dst, s);
            if (last) {   // the other two terms in their own tensors, added at the end
              launch_chain_f64(cd, (const double*)dcsrc, (const double*)c->dU64.p + u_off[j], d2Tn2 + slab, s);
              launch_chain_f64(cd, (const double*)csrc, (const double*)c->d2U64.p + u_off[j], d2Tn3 + slab, s);
            } else {
              launch_chain_f64(cd, (const double*)dcsrc, (const double*)c->dU64.p + u_off[j], tdst, s);
              launch_axpby(2.0, tdst, 1.0, d2dst, view_elems(out), s);
              launch_chain_f64(cd, (const double*)csrc, (const double*)c->d2U64.p + u_off[j], tdst, s);
              launch_axpby(1.0, tdst, 1.0, d2dst, view_elems(out), s);
            }
            d2csrc = d2dst;
          }
          dcsrc = ddst;
        }
      } else if (c->f64_chains && !tangent) {
        launch_chain_f64acc(cd, csrc, j == d - 1 ? 0 : 1, (const double*)c->U64.p + u_off[j], dst, OUT_F64, s);
      } else if (zfold && j == d - 1) {
        const Z2Chunk& ch = zch[n1lo / n1_chunk];
        Z2In zi;
        zi.rblk = zmap + moff_rowblk;
        zi.rpos = zmap + moff_rowpos;
        zi.cblk = zmap + ch.off_blk;
        zi.cpos = zmap + ch.off_pos;
        zi.q = c->par[to[0]][sl];
        zi.c[0] = (const float*)cblk_cur[0];
        zi.c[1] = (const float*)cblk_cur[1];
        zi.ld = ldz;
        tuned_chain(c, cd, 2, [&] { launch_chain_f32_z2in(cd, zi, (const float*)c->U32.p + u_off[j], dst, last ? OUT_F64 : OUT_F32, s); });
      } else {
        launch_chain_f32(cd, csrc, 0, (const float*)c->U32.p + u_off[j], dst, last ? OUT_F64 : OUT_F32, s);
        if (tangent) {   // the same in FP32 (FP64 output of the last stage)
          const long long slab = (long long)sl * Pn + (long long)n1lo * prod_after(nnew, 1);
          void* ddst = last ? (void*)(dTn + slab) : ((j & 1) ? c->dchA.p : c->dchB.p);
          void* tdst = last ? (void*)(dTn2 + slab) : c->dchT.p;
          const int mode = last ? OUT_F64 : OUT_F32;
          launch_chain_f32(cd, dcsrc, 0, (const float*)c->U32.p + u_off[j], ddst, mode, s);
          launch_chain_f32(cd, csrc, 0, (const float*)c->dU32.p + u_off[j], tdst, mode, s);
          if (!last) launch_add_f32((const float*)tdst, (float*)ddst, view_elems(out), s);
          dcsrc = ddst;
        }
      }
      csrc = dst;
      cin = out;
    }
  }
  }   // PH_FULL, PH_CONTRACT: the contraction

  if (phase == PH_CONTRACT) {
    // out: slice c' of T' (columns c' Pn .. of every row) at (c' - c_lo) Rn Pn, row-major
    if (pending_error(c, "the non-prime chain") != HOTRG_OK) return HOTRG_ECUDA;
    for (int sl = sl_lo; sl < sl_hi; ++sl)
      if (cudaMemcpy2DAsync(sh.out + (long long)(sl - sl_lo) * slice_elems, sizeof(double) * Pn,
                            Tn + (long long)sl * Pn, sizeof(double) * Rn, sizeof(double) * Pn, Rn,
                            cudaMemcpyDefault, s) != cudaSuccess)
        return cuda_status(c) == HOTRG_OK ? (c->poisoned = HOTRG_ECUDA) : HOTRG_ECUDA;
    c->shard_bn_done = bn_done;
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_status(c);
    return cuda_status(c);
  }
  if (phase == PH_FINISH) {
    // in: every slice, gathered over the ranks, in the layout PH_CONTRACT writes
    for (int sl = 0; sl < chi_c; ++sl)
      if (cudaMemcpy2DAsync(Tn + (long long)sl * Pn, sizeof(double) * Rn, sh.in + (long long)sl * slice_elems,
                            sizeof(double) * Pn, sizeof(double) * Pn, Rn, cudaMemcpyDefault, s) != cudaSuccess)
        return cuda_status(c) == HOTRG_OK ? (c->poisoned = HOTRG_ECUDA) : HOTRG_ECUDA;
    bn_done = c->shard_bn_done;   // this rank's share of the bottleneck
    c->shard_ready = 0;
  }

  if (pending_error(c, "the non-prime chain") != HOTRG_OK) return HOTRG_ECUDA;
  if (tangent) launch_axpby(1.0, dTn2, 1.0, dTn, Rn * Rn, s);
  if (tan2) {
    launch_axpby(2.0, d2Tn2, 1.0, d2Tn, Rn * Rn, s);
    launch_axpby(1.0, d2Tn3, 1.0, d2Tn, Rn * Rn, s);
  }
  // ---- bond dims of the new tensor (Sec. 4.2.15 with the axes kept physical)
  for (int j = 1; j < d; ++j) c->chis[to[j]] = nnew[j];
  if (track)
    for (int j = 1; j < d; ++j) c->par[to[j]] = newpar[j];
  c->last_z2 = z2 ? 1 : 0;
  c->last_bn_dense = bn_flops;
  c->last_bn_done = bn_done;
  c->p += 1;
  // ---- trace, Y, ratio X, ln Z, normalisation (Secs. 4.2.11-4.2.16)
  CHECK_ALLOC(dev_alloc(c, c->T, sizeof(double) * Rn * Rn));
  {
    Phase ph(c, 8);
    trace_and_normalise(c, Tn, 0);
    if (tangent) {
      CHECK_ALLOC(dev_alloc(c, c->dT, sizeof(double) * Rn * Rn));
      tangent_trace_and_normalise(c, dTn, 0);
    }
    if (tan2) {
      CHECK_ALLOC(dev_alloc(c, c->d2T, sizeof(double) * Rn * Rn));
      tangent2_trace_and_normalise(c, d2Tn, dTn, 0);
    }
  }

  c->last_valid = 1;
  c->last_nlegs = nlegs;
  for (int j = 1; j < d; ++j) {
    c->last_leg_axis[j - 1] = to[j];
    c->last_leg_n[j - 1] = chij[j] * chij[j];
    c->last_leg_nnew[j - 1] = nnew[j];
    c->last_lam_off[j - 1] = lam_off[j];
    c->last_u_off[j - 1] = u_off[j];
  }
  return cuda_status(c);
}

}  // namespace

int hotrg_shard_env(hotrg_ctx* c, int axis, int chi, int part, int nparts, double* S, int64_t cap,
                    int64_t* n) {
  if (nparts < 1 || part < 0 || part >= nparts) return HOTRG_EINVAL;
  Shard sh;
  sh.phase = PH_ENV;
  sh.part = part;
  sh.nparts = nparts;
  sh.out = S;
  sh.cap = cap;
  sh.n_out = n;
  return step_impl(c, axis, chi, sh);
}

int hotrg_shard_isometries(hotrg_ctx* c, int axis, int chi, const double* S, int64_t n) {
  Shard sh;
  sh.phase = PH_ISO;
  sh.in = S;
  sh.cap = n;
  return step_impl(c, axis, chi, sh);
}

int hotrg_shard_contract(hotrg_ctx* c, int axis, int chi, int c_lo, int c_hi, double* slices, int64_t cap,
                         int64_t* n) {
  Shard sh;
  sh.phase = PH_CONTRACT;
  sh.c_lo = c_lo;
  sh.c_hi = c_hi;
  sh.out = slices;
  sh.cap = cap;
  sh.n_out = n;
  return step_impl(c, axis, chi, sh);
}

int hotrg_shard_finish(hotrg_ctx* c, int axis, int chi, const double* slices, int64_t n) {
  Shard sh;
  sh.phase = PH_FINISH;
  sh.in = slices;
  sh.cap = n;
  return step_impl(c, axis, chi, sh);
}

static int find_leg(hotrg_ctx* c, int leg) {
  if (!c->last_valid) return -1;
  for (int j = 0; j < c->last_nlegs; ++j)
    if (c->last_leg_axis[j] == leg) return j;
  return -1;
}

int hotrg_isometry(hotrg_ctx* c, int leg, double* U, int64_t cap, int* rows, int* cols,
                   int* chosen_prime) {
  if (!c) return HOTRG_EINVAL;
  int r = sync_and_status(c, nullptr);
  if (r != HOTRG_OK) return r;
  int j = find_leg(c, leg);
  if (j < 0) return c->last_valid ? HOTRG_EINVAL : HOTRG_ESTATE;
  int n = c->last_leg_n[j], nn = c->last_leg_nnew[j];
  if (rows) *rows = n;
  if (cols) *cols = nn;
  LegResult lr;
  if (cudaMemcpy(&lr, (LegResult*)c->legres.p + (j + 1), sizeof(lr), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_status(c);
  if (chosen_prime) *chosen_prime = lr.chose_prime;
  if (!U || cap < (int64_t)n * nn) return HOTRG_EINVAL;
  if (cudaMemcpy(U, (double*)c->U64.p + c->last_u_off[j], sizeof(double) * n * nn, cudaMemcpyDefault) != cudaSuccess)
    return cuda_status(c);
  return HOTRG_OK;
}

int hotrg_spectrum(hotrg_ctx* c, int leg, int prime, double* lam, int64_t cap, int* n_out) {
  if (!c || (prime != 0 && prime != 1)) return HOTRG_EINVAL;
  int r = sync_and_status(c, nullptr);
  if (r != HOTRG_OK) return r;
  int j = find_leg(c, leg);
  if (j < 0) return c->last_valid ? HOTRG_EINVAL : HOTRG_ESTATE;
  int n = c->last_leg_n[j];
  if (n_out) *n_out = n;
  if (!lam || cap < n) return HOTRG_EINVAL;
  if (cudaMemcpy(lam, (double*)c->lam.p + c->last_lam_off[j] + (long long)prime * n, sizeof(double) * n,
                 cudaMemcpyDefault) != cudaSuccess)
    return cuda_status(c);
  return HOTRG_OK;
}

int hotrg_jacobi_sweeps(hotrg_ctx* c, int leg, int* sweeps) {
  if (!c || !sweeps) return HOTRG_EINVAL;
  int r = sync_and_status(c, nullptr);
  if (r != HOTRG_OK) return r;
  int j = find_leg(c, leg);
  if (j < 0) return c->last_valid ? HOTRG_EINVAL : HOTRG_ESTATE;
  LegResult lr;
  if (cudaMemcpy(&lr, (LegResult*)c->legres.p + (j + 1), sizeof(lr), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_status(c);
  *sweeps = lr.sweeps[0];
  return HOTRG_OK;
}

int hotrg_truncation(hotrg_ctx* c, int leg, double* eps, double* eps_prime) {
  if (!c) return HOTRG_EINVAL;
  int r = sync_and_status(c, nullptr);
  if (r != HOTRG_OK) return r;
  int j = find_leg(c, leg);
  if (j < 0) return c->last_valid ? HOTRG_EINVAL : HOTRG_ESTATE;
  LegResult lr;
  if (cudaMemcpy(&lr, (LegResult*)c->legres.p + (j + 1), sizeof(lr), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_status(c);
  if (eps) *eps = lr.eps[0];
  if (eps_prime) *eps_prime = lr.eps[1];
  return HOTRG_OK;
}

int hotrg_free_energy(hotrg_ctx* c, double* lnZ_per_site, double* f_per_site) {
  if (!c) return HOTRG_EINVAL;
  DevState st;
  int r = sync_and_status(c, &st);
  if (r != HOTRG_OK) return r;
  if (lnZ_per_site) *lnZ_per_site = st.ln_z_site;
  if (f_per_site) *f_per_site = c->beta > 0 ? -st.ln_z_site / c->beta : NAN;
  return HOTRG_OK;
}

int hotrg_observables(hotrg_ctx* c, double* trace, double* gu_wen_X, int* nsteps) {
  if (!c) return HOTRG_EINVAL;
  DevState st;
  int r = sync_and_status(c, &st);
  if (r != HOTRG_OK) return r;
  if (trace) *trace = st.trace;
  if (gu_wen_X) *gu_wen_X = st.gu_wen;
  if (nsteps) *nsteps = c->p;
  return HOTRG_OK;
}

int hotrg_bond_dims(hotrg_ctx* c, int dims[4]) {
  if (!c || !dims) return HOTRG_EINVAL;
  for (int k = 0; k < 4; ++k) dims[k] = k < c->d ? c->chis[k] : 0;
  return HOTRG_OK;
}

int hotrg_tensor(hotrg_ctx* c, double* T, int64_t cap, int dims[8]) {
  if (!c) return HOTRG_EINVAL;
  int r = sync_and_status(c, nullptr);
  if (r != HOTRG_OK) return r;
  long long n = tensor_elems(c);
  if (dims)
    for (int k = 0; k < 8; ++k) dims[k] = k < 2 * c->d ? c->chis[k / 2] : 0;
  if (!T || cap < n) return HOTRG_EINVAL;
  int ra = dev_alloc(c, c->Xp, sizeof(double) * n);
  if (ra != HOTRG_OK) return ra;
  slots_to_interchange(c, (const double*)c->T.p, (double*)c->Xp.p);
  if (cudaMemcpyAsync(T, c->Xp.p, sizeof(double) * n, cudaMemcpyDefault, c->stream) != cudaSuccess)
    return cuda_status(c);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_status(c);
  return cuda_status(c);
}

int hotrg_gemm_nt(int mode, int M, int N, int K, const double* A, const double* B, double* C) {
  if (mode < HOTRG_PREC_FP64 || mode > HOTRG_PREC_TF32X3 || M < 1 || N < 1 || K < 1 ||
      M > (1 << 20) || N > (1 << 20) || K > (1 << 20) || !A || !B || !C)
    return HOTRG_EINVAL;
  if ((long long)M * K > (1LL << 31) || (long long)N * K > (1LL << 31) || (long long)M * N > (1LL << 31))
    return HOTRG_EINVAL;
  if (mode != HOTRG_PREC_FP64 && !tc_gemm_ready()) return HOTRG_ECUDA;
  cudaStream_t s = nullptr;
  const int np = split_pieces(mode), pfmt = split_format(mode);
  const long long pbytes = piece_bytes(pfmt);
  const long long Kpad = mode == HOTRG_PREC_FP64 ? K : ((long long)K + 63) / 64 * 64;
  void *dA = nullptr, *dB = nullptr, *dC = nullptr, *pA = nullptr, *pB = nullptr, *c32 = nullptr;
  int* err = nullptr;
  int status = HOTRG_OK;
  auto fail = [&](int st) {
    if (status == HOTRG_OK) status = st;
  };
  if (cudaMalloc(&dA, sizeof(double) * M * K) || cudaMalloc(&dB, sizeof(double) * N * K) ||
      cudaMalloc(&dC, sizeof(double) * M * N) || cudaMalloc(&err, sizeof(int)))
    fail(HOTRG_ENOMEM);
  if (status == HOTRG_OK && mode != HOTRG_PREC_FP64) {
    if (cudaMalloc(&pA, pbytes * np * M * Kpad) || cudaMalloc(&pB, pbytes * np * N * Kpad) ||
        cudaMalloc(&c32, sizeof(float) * M * N))
      fail(HOTRG_ENOMEM);
  }
  if (status == HOTRG_OK) {
    cudaMemcpy(dA, A, sizeof(double) * M * K, cudaMemcpyDefault);
    cudaMemcpy(dB, B, sizeof(double) * N * K, cudaMemcpyDefault);
    cudaMemset(err, 0, sizeof(int));
    if (mode == HOTRG_PREC_FP64) {
      launch_gemm_nt_f64((const double*)dA, K, (const double*)dB, K, (double*)dC, N, 0, M, N, K, 1, 0, s);
    } else {
      cudaMemset(pA, 0, pbytes * np * M * Kpad);
      cudaMemset(pB, 0, pbytes * np * N * Kpad);
      launch_split((const double*)dA, M, K, K, pA, Kpad, M * Kpad, np, pfmt, s);
      launch_split((const double*)dB, N, K, K, pB, Kpad, N * Kpad, np, pfmt, s);
      int ta[6], tb[6];
      const int nt = split_terms(np, ta, tb);
      if (launch_tc_gemm(pA, M, pB, N, (int)Kpad, np, nt, ta, tb, (float*)c32, N, err, s, nullptr, pfmt) != 0)
        fail(HOTRG_ECUDA);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) fail(HOTRG_ECUDA);
    int e = 0;
    cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e) fail(e);
    if (status == HOTRG_OK) {
      if (mode == HOTRG_PREC_FP64) {
        cudaMemcpy(C, dC, sizeof(double) * M * N, cudaMemcpyDefault);
      } else {
        std::vector<float> h((size_t)M * N);
        cudaMemcpy(h.data(), c32, sizeof(float) * M * N, cudaMemcpyDeviceToHost);
        std::vector<double> hd(h.begin(), h.end());
        cudaMemcpy(C, hd.data(), sizeof(double) * M * N, cudaMemcpyDefault);
      }
      if (cudaGetLastError() != cudaSuccess) fail(HOTRG_ECUDA);
    }
  }
  cudaGetLastError();
  for (void* p : {dA, dB, dC, pA, pB, c32, (void*)err})
    if (p) cudaFree(p);
  return status;
}

// ---------------------------------------------------------------------------
// Captured steps (CUDA graph): the host state a step changes, so that a capture can
// be undone and a replay can apply it
// ---------------------------------------------------------------------------
namespace {
struct HostSnap {
  int p, last_fp64, last_valid, last_nlegs, last_z2, poisoned;
  int chis[kMaxD], order[kMaxD];
  int last_leg_axis[kMaxD - 1], last_leg_n[kMaxD - 1], last_leg_nnew[kMaxD - 1];
  long long last_lam_off[kMaxD - 1], last_u_off[kMaxD - 1];
  double last_bn_dense, last_bn_done;
  Buf T, T2;
};

HostSnap take_snap(const hotrg_ctx* c) {
  HostSnap h;
  h.p = c->p;
  h.last_fp64 = c->last_fp64;
  h.last_valid = c->last_valid;
  h.last_nlegs = c->last_nlegs;
  h.last_z2 = c->last_z2;
  h.poisoned = c->poisoned;
  for (int k = 0; k < kMaxD; ++k) {
    h.chis[k] = c->chis[k];
    h.order[k] = c->order[k];
  }
  for (int k = 0; k < kMaxD - 1; ++k) {
    h.last_leg_axis[k] = c->last_leg_axis[k];
    h.last_leg_n[k] = c->last_leg_n[k];
    h.last_leg_nnew[k] = c->last_leg_nnew[k];
    h.last_lam_off[k] = c->last_lam_off[k];
    h.last_u_off[k] = c->last_u_off[k];
  }
  h.last_bn_dense = c->last_bn_dense;
  h.last_bn_done = c->last_bn_done;
  h.T = c->T;
  h.T2 = c->T2;
  return h;
}

// the step count and the records of the last step
void put_step_records(hotrg_ctx* c, const HostSnap& h) {
  c->p = h.p;
  c->last_fp64 = h.last_fp64;
  c->last_valid = h.last_valid;
  c->last_nlegs = h.last_nlegs;
  c->last_z2 = h.last_z2;
  for (int k = 0; k < kMaxD - 1; ++k) {
    c->last_leg_axis[k] = h.last_leg_axis[k];
    c->last_leg_n[k] = h.last_leg_n[k];
    c->last_leg_nnew[k] = h.last_leg_nnew[k];
    c->last_lam_off[k] = h.last_lam_off[k];
    c->last_u_off[k] = h.last_u_off[k];
  }
  c->last_bn_dense = h.last_bn_dense;
  c->last_bn_done = h.last_bn_done;
}

bool same_layout(const hotrg_ctx* c, const HostSnap& h) {
  for (int k = 0; k < kMaxD; ++k)
    if (c->chis[k] != h.chis[k] || c->order[k] != h.order[k]) return false;
  return c->T.p == h.T.p && c->T2.p == h.T2.p;
}

// a context whose steps may be captured: no derivative, no parity read-back, no
// phase timing, no shard in progress
int capture_ready(const hotrg_ctx* c) {
  if (c->poisoned) return HOTRG_ESTATE;
  if (c->tangent || c->z2_valid || c->profile || c->shard_ready) return HOTRG_ESTATE;
  return HOTRG_OK;
}
}  // namespace

struct hotrg_graph {
  hotrg_ctx* owner = nullptr;
  cudaGraphExec_t exec = nullptr;
  int nsteps = 0;
  long long launches = 0;   // kernels of one replay
  HostSnap after;           // the host state the captured steps leave
};

int hotrg_graph_capture(hotrg_ctx* c, int n, const int* axes, int chi, hotrg_graph** out) {
  if (!c || !out || n < 1 || n > 64 || !axes || chi < 1 || chi > 32) return HOTRG_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (axes[i] < 0 || axes[i] >= c->d) return HOTRG_EINVAL;
  int r = capture_ready(c);
  if (r != HOTRG_OK) return r;
  if (pending_error(c, "work before the capture") != HOTRG_OK) return HOTRG_ECUDA;
  // the legacy default stream cannot be captured: record on a stream of our own
  cudaStream_t user_stream = c->stream, cs = c->stream;
  if (cs == nullptr && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_status(c);
  if (cudaStreamSynchronize(user_stream) != cudaSuccess) {
    if (cs != user_stream) cudaStreamDestroy(cs);
    return cuda_status(c);
  }
  const HostSnap before = take_snap(c);
  const long long launches0 = g_launches;
  c->stream = cs;
  c->capturing = 1;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    r = HOTRG_ECUDA;
  } else {
    for (int i = 0; i < n && r == HOTRG_OK; ++i) r = step_impl(c, axes[i], chi, Shard());
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (r == HOTRG_OK && e != cudaSuccess) r = HOTRG_ECUDA;
  }
  c->capturing = 0;
  c->stream = user_stream;
  const long long captured = g_launches - launches0;
  g_launches -= captured;   // nothing ran
  const HostSnap after = take_snap(c);
  // nothing of the captured steps ran: put the host state back
  put_step_records(c, before);
  for (int k = 0; k < kMaxD; ++k) {
    c->chis[k] = before.chis[k];
    c->order[k] = before.order[k];
  }
  c->T = before.T;
  c->T2 = before.T2;
  c->poisoned = before.poisoned;
  cudaGetLastError();   // a refused capture leaves its error here
  if (cs != user_stream) cudaStreamDestroy(cs);
  // the sequence must end where it starts (bond dims, slot order, buffers), so that it
  // can be replayed back to back
  if (r == HOTRG_OK) {
    bool closed = true;
    for (int k = 0; k < kMaxD; ++k)
      closed = closed && after.chis[k] == before.chis[k] && after.order[k] == before.order[k];
    closed = closed && after.T.p == before.T.p && after.T2.p == before.T2.p;
    if (!closed) r = HOTRG_ESTATE;
  }
  cudaGraphExec_t exec = nullptr;
  if (r == HOTRG_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    r = HOTRG_ECUDA;
  }
  if (graph) cudaGraphDestroy(graph);
  if (r != HOTRG_OK) return r;
  hotrg_graph* g = new hotrg_graph();
  g->owner = c;
  g->exec = exec;
  g->nsteps = n;
  g->launches = captured;
  g->after = after;
  *out = g;
  return HOTRG_OK;
}

int hotrg_graph_launch(hotrg_ctx* c, hotrg_graph* g) {
  if (!c || !g || g->owner != c) return HOTRG_EINVAL;
  int r = capture_ready(c);
  if (r != HOTRG_OK) return r;
  if (!same_layout(c, g->after)) return HOTRG_ESTATE;   // not at the start of the captured cycle
  if (cudaGraphLaunch(g->exec, c->stream) != cudaSuccess) {
    cuda_status(c);
    return HOTRG_ECUDA;
  }
  g_launches += g->launches;
  HostSnap rec = g->after;
  rec.p = c->p + g->nsteps;
  put_step_records(c, rec);
  return pending_error(c, "the graph launch");
}

void hotrg_graph_free(hotrg_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
}

int hotrg_step_batch(hotrg_ctx** ctxs, int n, const int* axes, const int* chis, int nthreads,
                     int* status) {
  if (n < 0 || (n > 0 && (!ctxs || !axes || !chis))) return HOTRG_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return HOTRG_EINVAL;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return HOTRG_EINVAL;   // one thread per context at a time
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  nthreads = std::min(nthreads, std::max(n, 1));
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<int> st(n, HOTRG_OK);
  std::atomic<int> next{0};
  auto work = [&]() {
    cudaSetDevice(dev);
    for (int i = next++; i < n; i = next++) st[i] = hotrg_step(ctxs[i], axes[i], chis[i]);
  };
  std::vector<std::thread> pool;
  try {
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(work);
  } catch (const std::system_error&) {
    // no more threads to be had: the ones started (and this one) take every context
  }
  work();
  for (auto& th : pool) th.join();
  int first = HOTRG_OK;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = st[i];
    if (first == HOTRG_OK) first = st[i];
  }
  return first;
}

int hotrg_set_z2(hotrg_ctx* c, int enable) {
  if (!c) return HOTRG_EINVAL;
  c->z2_enabled = enable ? 1 : 0;
  return HOTRG_OK;
}

int hotrg_set_parity(hotrg_ctx* c, const int* parity) {
  if (!c) return HOTRG_EINVAL;
  if (c->poisoned) return HOTRG_ESTATE;
  if (!parity) {   // forget them: dense steps from here on, with no read-back
    c->z2_valid = 0;
    for (int k = 0; k < kMaxD; ++k) c->par[k].clear();
    return HOTRG_OK;
  }
  const int d = c->d;
  std::vector<unsigned char> par[kMaxD];
  int off = 0;
  for (int k = 0; k < d; ++k) {
    for (int v = 0; v < c->chis[k]; ++v) {
      const int x = parity[off + v];
      if (x != 0 && x != 1) return HOTRG_EINVAL;
      par[k].push_back((unsigned char)x);
    }
    off += c->chis[k];
  }
  Z2Slots sl;
  sl.d = d;
  for (int k = 0; k < d; ++k) {
    const int ax = c->order[k];
    sl.chi[k] = c->chis[ax];
    sl.mask[k] = 0;
    for (int v = 0; v < c->chis[ax]; ++v) sl.mask[k] |= (unsigned)par[ax][v] << v;
  }
  CHECK_ALLOC(dev_alloc(c, c->counters, sizeof(int) * kCounterInts));
  int* cnt = (int*)c->counters.p;
  int bad = 0;
  cudaMemsetAsync(cnt, 0, sizeof(int), c->stream);
  launch_z2_check((const double*)c->T.p, sl, tensor_elems(c), cnt, c->stream);
  if (cudaMemcpyAsync(&bad, cnt, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return cuda_status(c);
  if (bad) return HOTRG_EINVAL;
  for (int k = 0; k < d; ++k) c->par[k] = par[k];
  c->z2_valid = 1;
  return HOTRG_OK;
}

int hotrg_leg_parity(hotrg_ctx* c, int* parity, int cap, int* n_out) {
  if (!c || !parity) return HOTRG_EINVAL;
  if (!c->z2_valid) return HOTRG_ESTATE;
  int n = 0;
  for (int k = 0; k < c->d; ++k) n += c->chis[k];
  if (n_out) *n_out = n;
  if (cap < n) return HOTRG_EINVAL;
  int off = 0;
  for (int k = 0; k < c->d; ++k)
    for (int v = 0; v < c->chis[k]; ++v) parity[off++] = c->par[k][v];
  return HOTRG_OK;
}

int hotrg_bottleneck_flops(hotrg_ctx* c, double* dense, double* performed, int* z2_blocks) {
  if (!c) return HOTRG_EINVAL;
  if (!c->last_valid) return HOTRG_ESTATE;
  if (dense) *dense = c->last_bn_dense;
  if (performed) *performed = c->last_bn_done;
  if (z2_blocks) *z2_blocks = c->last_z2;
  return HOTRG_OK;
}

int hotrg_set_tangent(hotrg_ctx* c, int enable) {
  if (!c || enable < 0 || enable > 2) return HOTRG_EINVAL;
  if (!enable) {
    c->tangent = 0;
    return HOTRG_OK;
  }
  if (c->poisoned) return HOTRG_ESTATE;
  if (c->tangent == enable) return HOTRG_OK;
  if (!c->is_ising || c->p != 0 || !(c->beta > 0.0)) return HOTRG_EINVAL;
  if (enable == 2 && c->precision != HOTRG_PREC_FP64) return HOTRG_EINVAL;   // second order: FP64 form
  const long long n = tensor_elems(c);
  CHECK_ALLOC(dev_alloc(c, c->tstate, sizeof(TanState)));
  CHECK_ALLOC(dev_alloc(c, c->Yd, sizeof(double) * kMaxBond * kMaxBond));
  CHECK_ALLOC(dev_alloc(c, c->dT2, sizeof(double) * n));
  CHECK_ALLOC(dev_alloc(c, c->dT, sizeof(double) * n));
  cudaMemsetAsync(c->tstate.p, 0, sizeof(TanState), c->stream);
  launch_init_ising_dbeta((double*)c->dT2.p, c->d, c->beta, c->h, c->stream);
  tangent_trace_and_normalise(c, (const double*)c->dT2.p, 1);
  if (enable == 2) {
    CHECK_ALLOC(dev_alloc(c, c->Yd2, sizeof(double) * kMaxBond * kMaxBond));
    CHECK_ALLOC(dev_alloc(c, c->d2T2, sizeof(double) * n));
    CHECK_ALLOC(dev_alloc(c, c->d2T, sizeof(double) * n));
    launch_init_ising_d2beta((double*)c->d2T2.p, c->d, c->beta, c->h, c->stream);
    tangent2_trace_and_normalise(c, (const double*)c->d2T2.p, (const double*)c->dT2.p, 1);
  }
  c->tangent = enable;
  return cuda_status(c);
}

int hotrg_specific_heat(hotrg_ctx* c, double* d2lnz_dbeta2, double* specific_heat) {
  if (!c) return HOTRG_EINVAL;
  if (c->tangent != 2) return HOTRG_ESTATE;
  int r = sync_and_status(c, nullptr);
  if (r != HOTRG_OK) return r;
  TanState t;
  if (cudaMemcpy(&t, c->tstate.p, sizeof(t), cudaMemcpyDeviceToHost) != cudaSuccess) return cuda_status(c);
  if (d2lnz_dbeta2) *d2lnz_dbeta2 = t.d2ln_z_site;
  if (specific_heat) *specific_heat = c->beta * c->beta * t.d2ln_z_site;
  return HOTRG_OK;
}

int hotrg_energy(hotrg_ctx* c, double* dlnz_dbeta, double* energy, int* degenerate_pairs) {
  if (!c) return HOTRG_EINVAL;
  if (!c->tangent) return HOTRG_ESTATE;
  int r = sync_and_status(c, nullptr);
  if (r != HOTRG_OK) return r;
  TanState t;
  if (cudaMemcpy(&t, c->tstate.p, sizeof(t), cudaMemcpyDeviceToHost) != cudaSuccess) return cuda_status(c);
  if (dlnz_dbeta) *dlnz_dbeta = t.dln_z_site;
  if (energy) *energy = -t.dln_z_site;
  if (degenerate_pairs) *degenerate_pairs = t.degenerate;
  return HOTRG_OK;
}

int hotrg_tangent_tensor(hotrg_ctx* c, double* dT, int64_t cap, int dims[8]) {
  if (!c) return HOTRG_EINVAL;
  if (!c->tangent) return HOTRG_ESTATE;
  int r = sync_and_status(c, nullptr);
  if (r != HOTRG_OK) return r;
  long long n = tensor_elems(c);
  if (dims)
    for (int k = 0; k < 8; ++k) dims[k] = k < 2 * c->d ? c->chis[k / 2] : 0;
  if (!dT || cap < n) return HOTRG_EINVAL;
  int ra = dev_alloc(c, c->Xp, sizeof(double) * n);
  if (ra != HOTRG_OK) return ra;
  slots_to_interchange(c, (const double*)c->dT.p, (double*)c->Xp.p);
  if (cudaMemcpyAsync(dT, c->Xp.p, sizeof(double) * n, cudaMemcpyDefault, c->stream) != cudaSuccess)
    return cuda_status(c);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_status(c);
  return cuda_status(c);
}

int hotrg_set_fp64_threshold(hotrg_ctx* c, double flops) {
  if (!c || !(flops >= 0.0)) return HOTRG_EINVAL;
  c->fp64_below = flops;
  return HOTRG_OK;
}

int hotrg_set_slice_budget(hotrg_ctx* c, double bytes) {
  if (!c || !(bytes >= 0.0)) return HOTRG_EINVAL;
  c->slice_budget_bytes = bytes;
  return HOTRG_OK;
}

int hotrg_profile(hotrg_ctx* c, int enable) {
  if (!c || enable < 0 || enable > 2) return HOTRG_EINVAL;
  c->profile = enable;
  c->marks.clear();
  c->event_next = 0;
  return HOTRG_OK;
}

int hotrg_step_times(hotrg_ctx* c, double ms[16], int launches[16], int* n, int* contraction_fp64) {
  if (!c || !ms) return HOTRG_EINVAL;
  int r = sync_and_status(c, nullptr);
  if (r != HOTRG_OK) return r;
  for (int k = 0; k < 16; ++k) {
    ms[k] = 0.0;
    if (launches) launches[k] = 0;
  }
  for (auto& m : c->marks) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, m.second.first, m.second.second) != cudaSuccess) return cuda_status(c);
    ms[m.first] += t;
    if (launches) launches[m.first] += 1;
  }
  if (c->profile == 2) {   // read once: start the next collection
    c->marks.clear();
    c->event_next = 0;
  }
  if (n) *n = 12;
  if (contraction_fp64) *contraction_fp64 = c->last_fp64;
  return HOTRG_OK;
}

int hotrg_gemm_rate(int mode, int M, int N, int K, int iters, double* ms_per_launch) {
  if (mode <= HOTRG_PREC_FP64 || mode > HOTRG_PREC_TF32X3 || M < 1 || N < 1 || K < 1 || M > (1 << 20) ||
      N > (1 << 20) || K > (1 << 20) || iters < 1 || !ms_per_launch)
    return HOTRG_EINVAL;
  if (!tc_gemm_ready()) return HOTRG_ECUDA;
  const int r = measure_tc_gemm_rate(split_pieces(mode), M, N, (K + 63) / 64 * 64, iters, ms_per_launch,
                                     split_format(mode));
  if (r == -1) return HOTRG_EINVAL;
  if (r == -2) return HOTRG_ENOMEM;
  if (r == -3) return HOTRG_ECUDA;
  return r;
}

int hotrg_fp64_rate(double* tflops) {
  if (!tflops) return HOTRG_EINVAL;
  const int r = measure_fp64_rate(tflops);
  return r == 0 ? HOTRG_OK : (r == -2 ? HOTRG_ENOMEM : HOTRG_ECUDA);
}

int hotrg_device_bytes(hotrg_ctx* c, size_t* bytes) {
  if (!c || !bytes) return HOTRG_EINVAL;
  *bytes = c->held;
  return HOTRG_OK;
}

int hotrg_launch_count(hotrg_ctx* c, int64_t* launches) {
  if (!c || !launches) return HOTRG_EINVAL;
  *launches = g_launches;
  return HOTRG_OK;
}

void hotrg_free(hotrg_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  cudaGetLastError();
  Buf* b[] = {&c->T,  &c->T2, &c->Xp,     &c->parts, &c->S,     &c->Amat,     &c->W,
              &c->V,  &c->lam, &c->U64,   &c->U32,   &c->legres, &c->Y,       &c->state,
              &c->counters, &c->sweeps, &c->Ap, &c->Bp, &c->Cb, &c->chA, &c->chB,
              &c->J32,  &c->Gns, &c->Vtmp, &c->Za, &c->Zb, &c->Zc, &c->Zmap, &c->Zg, &c->Eb,
              &c->dT, &c->dT2, &c->dTb, &c->dXp, &c->dS, &c->dA, &c->dU64, &c->eG, &c->eZ, &c->eZt,
              &c->rank, &c->Yd, &c->tstate, &c->dchA, &c->dchB, &c->dchT, &c->dBp, &c->tBp, &c->dCb,
              &c->tCb, &c->dAp, &c->dB64, &c->dU32, &c->d2T, &c->d2T2, &c->d2Tb, &c->d2Tc, &c->d2Xp,
              &c->d2S, &c->d2A, &c->d2U64, &c->eG1, &c->eW, &c->eZ2, &c->eZ2t, &c->d2chA, &c->d2chB,
              &c->d2Bp, &c->d2Cb, &c->Yd2, &c->parts2};
  for (auto* x : b) dev_release(c, *x);
  for (auto e : c->event_pool) cudaEventDestroy(e);
  for (auto e : c->tune_ev)
    if (e) cudaEventDestroy(e);
  if (c->hpin) cudaFreeHost(c->hpin);
  if (c->hpin_ev) cudaEventDestroy(c->hpin_ev);
  delete c;
}

}  // extern "C"
