/*
 * hotrg.h -- C ABI of the GB300 HOTRG coarse-graining library (libhotrg.so).
 *
 * Method: Yamashita & Sakurai, "A Parallel Computing Method for the Higher
 * Order Tensor Renormalization Group" (arXiv:2110.03607).  One call of
 * hotrg_step() is one coarse-graining along one lattice axis (Sec. 2, Eq.
 * CoarseGrainingProcedure_d; Sec. 4.2): environment matrices A^(j), A'^(j)
 * (Sec. 3.2), their eigen-decomposition (Sec. 4.2.5), the choice and
 * truncation of the isometries (Secs. 4.2.6-4.2.8), the contraction for the
 * new tensor (Sec. 4.2.9), and the trace / normalisation / ln Z bookkeeping
 * (Secs. 4.1.1, 4.2.11-4.2.16).  Everything after the argument checks runs
 * as CUDA kernels on one GPU; there is no CPU fallback.
 *
 * Conventions
 *  - Every function returns a status (HOTRG_OK or a negative HOTRG_E*);
 *    outputs go through out-pointers.  hotrg_strerror() names a status.
 *  - The library owns all device memory of a context.  It allocates with
 *    cudaMalloc, or through the hook given to hotrg_set_allocator().
 *  - hotrg_step() only enqueues work on the context's stream and returns,
 *    except that while the leg parities are known (hotrg_set_z2) it waits
 *    once per step for the isometries, whose column parities give the new
 *    legs' parities and shape the Z2 block form of the contraction, and
 *    that while a derivative is carried it waits for the per-leg choices.
 *    The read-back calls (hotrg_free_energy, hotrg_observables,
 *    hotrg_isometry, hotrg_spectrum, hotrg_tensor) synchronise that stream.
 *  - Device-side failures (a non-positive or non-finite trace, a Jacobi
 *    sweep cap, a bounded wait that expired) are recorded in a device status
 *    word and returned by the next read-back call.  After any failure other
 *    than HOTRG_EINVAL the context is poisoned: further calls return
 *    HOTRG_ESTATE until it is freed.
 *  - Tensor interchange layout: a local tensor of a d-dimensional lattice is
 *    a dense, row-major array with 2d axes (x_1, x_1', x_2, x_2', ...,
 *    x_d, x_d'), the index order of Eq. (2.4); axis k (0-based) has bond
 *    dimension dims[2k] = dims[2k+1].  Pointers passed for tensors may be
 *    host or device pointers (they are copied with cudaMemcpyDefault).
 *  - Lattice axes are 0-based: 0 = x, 1 = y, 2 = z, 3 = w.
 */
#ifndef HOTRG_H
#define HOTRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hotrg_ctx hotrg_ctx;

enum hotrg_status {
  HOTRG_OK = 0,
  HOTRG_EINVAL = -1,    /* bad argument or buffer too small (size out-params still set) */
  HOTRG_ENOMEM = -2,    /* device allocation failed */
  HOTRG_ECUDA = -3,     /* a CUDA runtime or driver call failed */
  HOTRG_ENUMERIC = -4,  /* trace of a new tensor <= 0 or not finite */
  HOTRG_ENOTCONV = -5,  /* Jacobi eigen-solver hit its sweep cap */
  HOTRG_ETIMEOUT = -6,  /* a bounded device-side wait expired */
  HOTRG_ESTATE = -7     /* context poisoned by an earlier failure, or no step yet */
};

/* Arithmetic of the contractions (prime chain, bottleneck, non-prime chain).
 * The environment matrices, the eigen-solver and the ln Z accumulation are
 * FP64 in every mode.  BF16X3: operands split into 2 BF16 pieces, 3 piece
 * products, FP32 accumulation.  BF16X6: 3 pieces, 6 products.  TF32: one TF32
 * piece (10 stored mantissa bits, rounded to nearest), one product.  TF32X3: 2
 * TF32 pieces, 3 products.  The tensor cores take TF32 at half the BF16 rate,
 * so TF32X3 issues as much tensor time as BF16X6.  FP64: plain FP64
 * everywhere. */
enum hotrg_precision {
  HOTRG_PREC_FP64 = 0,
  HOTRG_PREC_BF16X3 = 1,
  HOTRG_PREC_BF16X6 = 2,
  HOTRG_PREC_TF32 = 3,
  HOTRG_PREC_TF32X3 = 4
};

/* Start a run from the Ising initial tensor of Sec. 2, Eq. (2.4):
 * W_{s s'} = exp(beta s s'), X = U sqrt(Lambda), V_s = exp(beta h s),
 * sigma_0 = +1, sigma_1 = -1; bond dimension 2 on every leg.  The tensor is
 * normalised by f^(0) = 1/Tr T (Sec. 4.2.1) and ln Z^(0) = ln Tr T^(0).
 * d in [2, 4]; beta >= 0 (beta = 0 allowed; sqrt(sinh beta) is imaginary
 * for beta < 0).  On success *out owns a new context (default stream 0,
 * precision BF16X6).  At h = 0 the run starts with known leg parities
 * (index 0 even, index 1 odd; every element of odd total parity is zero) and
 * the contraction uses the Z2 block form of hotrg_set_z2.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int hotrg_init_ising(int d, double beta, double h, hotrg_ctx** out);

/* Start a run from a caller-given initial tensor T (interchange layout,
 * dims[2k] = dims[2k+1] = chis[k], 1 <= chis[k] <= 32).  Normalised as in
 * hotrg_init_ising.  beta is used only to report f = -(ln Z/V)/beta. */
int hotrg_init_tensor(int d, const int* chis, const double* T, double beta, hotrg_ctx** out);

/* Replace the current (normalised) local tensor of a run by T with bond
 * dimensions chis, keeping the run's K / ln Z bookkeeping (a resume from a
 * checkpoint).  The leg parities become unknown (see hotrg_set_parity).
 * Synchronous.  Errors: EINVAL, ENOMEM, ECUDA, ESTATE. */
int hotrg_set_tensor(hotrg_ctx* ctx, const int* chis, const double* T);

/* Use `stream` (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
 * for all later work of the context.  NULL = the legacy default stream. */
int hotrg_set_stream(hotrg_ctx* ctx, void* stream);

/* Route the context's device allocations through alloc/free (e.g. a caching
 * allocator).  alloc(bytes, user) returns a device pointer or NULL;
 * free(ptr, user) releases it.  Buffers already held are released through
 * the previous allocator first.  Pass NULL, NULL to return to cudaMalloc. */
typedef void* (*hotrg_alloc_fn)(size_t bytes, void* user);
typedef void (*hotrg_free_fn)(void* ptr, void* user);
int hotrg_set_allocator(hotrg_ctx* ctx, hotrg_alloc_fn alloc, hotrg_free_fn free_fn, void* user);

/* Select the contraction arithmetic (enum hotrg_precision). */
int hotrg_set_precision(hotrg_ctx* ctx, int mode);

/* In the BF16 modes, run the contraction of a step in FP64 when its
 * bottleneck needs fewer than `flops` floating-point operations (the early
 * steps of a run, while the bonds grow: they are cheap, and an error made
 * in step p weighs 2^-p in ln Z / V).  Default 2^36; 0 = never. */
int hotrg_set_fp64_threshold(hotrg_ctx* ctx, double flops);

/* Cap, in bytes, on the device memory of the per-slice contraction operands
 * (bottleneck operand pieces, its FP32 product, chain intermediates).  Each
 * c'-slice of the new-tensor contraction (Sec. 4.2.9) is further cut into
 * sub-ranges of n'_1 so that one sub-range fits the smaller of this cap and
 * 60 % of the free device memory.  Default 160e9. */
int hotrg_set_slice_budget(hotrg_ctx* ctx, double bytes);

/* Z2 (spin-flip) block form of the new-tensor contraction; enable = 1 is the
 * default.  It applies while the leg parities are known: from
 * hotrg_init_ising at h = 0, or declared by hotrg_set_parity.  The Ising
 * tensor at h = 0 vanishes on odd total parity; every isometry column then
 * has a definite parity (checked each step on the host: a column whose
 * nonzero rows mix parities ends the block form for the rest of the run),
 * and the bottleneck of Eq. (BottleneckPart) reduces to two dense blocks per
 * c'-slice, a quarter of the dense flops; the environment Grams (Sec. 3.2)
 * are block diagonal in the same way and are computed as two blocks.  The
 * paper works densely; the result is the same up to rounding (products with
 * an exact-zero factor are dropped, partial sums grouped differently).  With
 * enable = 0 everything is dense and the parities are still tracked. */
int hotrg_set_z2(hotrg_ctx* ctx, int enable);

/* Launch-shape autotuner (the paper has no counterpart): with enable = 1, the
 * first launch of each chain-stage shape (the tensor-times-isometry stages of
 * Sec. 4.2.9 on the default paths) runs once per candidate grid cap (4, 8,
 * 16, 32 CTAs per SM) on the real operands, timed with CUDA events on the
 * context's stream (the host waits for those events: that step is not
 * asynchronous), and the fastest is kept for the shape in the context.  A
 * stage's output does not depend on its grid, so results are the same bit for
 * bit with or without it.  Cached choices stay in use after enable = 0 and in
 * captured graphs; a graph capture never tunes.  Errors: EINVAL. */
int hotrg_set_autotune(hotrg_ctx* ctx, int enable);

/* *n = number of tuned chain-stage shapes; their choices (CTAs per SM) go to
 * choices[0 .. *n) when choices is given.  Errors: EINVAL (cap < *n). */
int hotrg_autotune_entries(hotrg_ctx* ctx, int* n, int* choices, int cap);

/* Declare the parity (0 or 1) of every index of the current tensor:
 * `parity` holds chis[0] entries for axis 0, then chis[1] for axis 1, ...
 * (the two legs of an axis share them).  Checked on the device: if an
 * element of odd total parity is nonzero the call returns EINVAL and the
 * parities stay unknown.  Synchronous.  parity = NULL forgets the parities:
 * later steps are dense and read nothing back (so they can be captured,
 * hotrg_graph_capture).  Errors: EINVAL, ENOMEM, ECUDA, ESTATE. */
int hotrg_set_parity(hotrg_ctx* ctx, const int* parity);

/* Read the known leg parities back in the layout of hotrg_set_parity;
 * *n = number of entries (sum of the bond dimensions).  Errors: EINVAL (cap
 * < *n), ESTATE (parities unknown). */
int hotrg_leg_parity(hotrg_ctx* ctx, int* parity, int cap, int* n);

/* Floating-point operations of the last step's bottleneck (Eq.
 * BottleneckPart): *dense = 2 R^2 P_new P chi_c of the dense contraction,
 * *performed = those of the GEMMs actually launched (a quarter of that with
 * the Z2 block form, padding excluded); *z2_blocks = 1 if the block form
 * ran.  Errors: EINVAL, ESTATE (no step yet). */
int hotrg_bottleneck_flops(hotrg_ctx* ctx, double* dense, double* performed, int* z2_blocks);

/* Record CUDA events around the phases of every later step (enable = 1), around
 * the bottleneck GEMM launches only, summed over all steps until the next
 * hotrg_step_times() call (enable = 2: no per-step read-back needed), or stop
 * (0).  hotrg_step_times() then returns, after synchronising, the
 * milliseconds of the last step (enable = 1) per phase: [0] leg permutation, [1]
 * environment Grams and A assembly, [2] Jacobi, [3] choice/truncation,
 * [4] BF16 split of T, [5] prime-side chain, [6] bottleneck GEMM, [7]
 * non-prime chain, [8] trace / normalisation, [9] FP32 warm start of the
 * eigen-solver (included in [2]), [10] its FP32 sweeps (included in [9]),
 * [11] gathers and scatters of the Z2 block form; *n = 12.  launches[k] =
 * number of timed regions of phase k (the bottleneck: one GEMM launch per
 * c'-slice and n'_1 sub-range, two with the Z2 block form).
 * *contraction_fp64 = 1 if the last step's contraction ran in FP64. */
int hotrg_profile(hotrg_ctx* ctx, int enable);
int hotrg_step_times(hotrg_ctx* ctx, double ms[16], int launches[16], int* n, int* contraction_fp64);

/* One coarse-graining along lattice axis `axis` in [0, d) with bond-
 * dimension parameter chi >= 1 (Sec. 2: chi_j^new = min(chi_j^2, chi) on
 * every transverse leg j; the axis's own bond is unchanged).  Transverse
 * legs are labelled Next j = axis (axis + j) mod d (Sec. 3.1.2).  The new
 * tensor is normalised by 1/Tr (Secs. 4.2.14-4.2.16).  Asynchronous, with
 * two exceptions that wait for the stream up to the choice of the isometries:
 * a step that tracks Z2 leg parities (the block form at zero field) copies the
 * kept isometries (a few hundred KB) to the host to derive the new legs'
 * parities, and a step that carries a derivative reads the per-leg choices
 * back.  hotrg_set_parity(ctx, NULL) drops the parities (dense steps from then
 * on, no wait).  Errors: EINVAL (axis out of range, chi outside [1, 32]),
 * ENOMEM, ECUDA, ESTATE. */
int hotrg_step(hotrg_ctx* ctx, int axis, int chi);

/* Batching form: one coarse-graining step on each of n independent contexts
 * (e.g. a scan over beta, h and chi), ctxs[i] along axes[i] with chis[i].
 * Host threads (nthreads; <= 0: the hardware threads, at most n) each take the
 * next context in turn, so the host-side waits of one context (the Z2 parity
 * read-back) overlap the device work of the others; the contexts should have
 * their own streams (hotrg_set_stream), else their kernels serialise on the
 * shared stream.  Allocation hooks are called from these threads.  A context
 * may appear once.  Returns the first failing status in index order (status[i],
 * if given, receives each context's status).  Errors: EINVAL, and those of
 * hotrg_step. */
int hotrg_step_batch(hotrg_ctx** ctxs, int n, const int* axes, const int* chis, int nthreads,
                     int* status);

/* Captured steps (CUDA graph; the paper has no counterpart).  hotrg_graph_capture
 * records the n steps hotrg_step(ctx, axes[i], chi) would enqueue, without running
 * them, into one executable graph.  The sequence must be closed: after it the bond
 * dimensions, the slot order and the buffers of the tensor are those before it
 * (the tensor alternates between two buffers every step and the slot order turns
 * with the axis, so in steady state a closed sequence is lcm(2, d) steps of the
 * cyclic axes: 2 in 2D, 6 in 3D, 4 in 4D); else HOTRG_ESTATE and nothing is kept.
 * The context must be past bond growth and must have run the same steps once
 * uncaptured (its buffers are then in place: a step that would allocate returns
 * HOTRG_ESTATE), and must carry no derivative, no known leg parities (the Z2
 * parity read-back waits on the host: hotrg_set_parity(ctx, NULL) drops them),
 * no phase timing and no shard step.  The context's state is left as it was.
 * hotrg_graph_launch enqueues one replay on the context's stream (asynchronous)
 * and advances the run by n steps: the same kernels with the same arguments as
 * the uncaptured steps, so the results are the same bit for bit; the step
 * count of the ln Z bookkeeping is read on the device.  A graph belongs to its
 * context and may be launched only at the start of its cycle (ESTATE
 * otherwise); free it before the context.  Errors: EINVAL, ESTATE, ECUDA. */
typedef struct hotrg_graph hotrg_graph;
int hotrg_graph_capture(hotrg_ctx* ctx, int n, const int* axes, int chi, hotrg_graph** out);
int hotrg_graph_launch(hotrg_ctx* ctx, hotrg_graph* graph);
void hotrg_graph_free(hotrg_graph* graph);

/* c'-slice shard of one step over W ranks (processes, one GPU each), each holding
 * a context with the same local tensor (the paper's replication of T over its
 * processes, Secs. 3.2 and 4.2.3-4.2.4).  A step along `axis` with `chi` is:
 *   1. hotrg_shard_env(part = rank, nparts = W): this rank's share of every
 *      environment Gram S^, S~, S^', S~' of Sec. 3.2 -- the sum over its part of
 *      the summed index (the indices other than the free pair; of each Z2
 *      parity block when the block form applies) -- written to S.  Layout:
 *      transverse legs j = 1 .. d-1 of the step (lattice axis (axis + j) mod d),
 *      for each the kinds S^ (free n_j, c'), S~ (n_j, c), S^' (n'_j, c'),
 *      S~' (n'_j, c), each an m_j x m_j row-major FP64 matrix, m_j = chi_j chi_c,
 *      concatenated; *n = 4 sum_j m_j^2 elements (set even when cap is too small).
 *   2. the caller sums S over the ranks (an allreduce), then
 *      hotrg_shard_isometries(S, n) on every rank: A^(j), A'^(j) (Sec. 4.2.4),
 *      the eigen-solver (Sec. 4.2.5), the choice, truncation and gauge
 *      (Secs. 4.2.6-4.2.8) and, at zero field, the new legs' parities.  Equal
 *      summed Grams give every rank the same isometries.
 *   3. hotrg_shard_contract(c_lo, c_hi): the new tensor's c'-slices [c_lo, c_hi)
 *      (Sec. 4.2.9: prime chain, bottleneck, non-prime chain; no communication)
 *      into `slices`: slice c' is the block T'[(c, n)][(c', n')] for every row
 *      (c, n) and every n', Rn x Pn row-major (Rn = chi_c Pn, Pn = the product
 *      of the new transverse bond dimensions), at (c' - c_lo) Rn Pn; *n =
 *      (c_hi - c_lo) Rn Pn.
 *   4. the caller gathers the slices of all ranks in c' order (an allgather),
 *      then hotrg_shard_finish(slices, n = chi_c Rn Pn) on every rank: the new
 *      tensor is installed and the trace, Y, X, ln Z bookkeeping and
 *      normalisation of Secs. 4.1.1, 4.2.11-4.2.16 run as in hotrg_step.
 * Every call is synchronous (S and slices may be host or device pointers).
 * The result equals hotrg_step's up to the grouping of the Grams' sums.  Calls
 * out of order return ESTATE; a step that carries d/d beta cannot be sharded
 * (EINVAL).  Errors: EINVAL (bad part, range or size), ENOMEM, ECUDA, ESTATE,
 * and the device failures of hotrg_step. */
int hotrg_shard_env(hotrg_ctx* ctx, int axis, int chi, int part, int nparts, double* S, int64_t cap,
                    int64_t* n);
int hotrg_shard_isometries(hotrg_ctx* ctx, int axis, int chi, const double* S, int64_t n);
int hotrg_shard_contract(hotrg_ctx* ctx, int axis, int chi, int c_lo, int c_hi, double* slices,
                         int64_t cap, int64_t* n);
int hotrg_shard_finish(hotrg_ctx* ctx, int axis, int chi, const double* slices, int64_t n);

/* Differentiation form: carry dT = dT/d beta through every later step in
 * forward mode, so that hotrg_energy() returns d(ln Z/V)/d beta and the
 * internal energy u = -d(ln Z/V)/d beta of the HOTRG approximation (Sec. 2
 * model; the paper does not differentiate the method).  Per step: the
 * derivatives of the chosen environments, dS = dX X^T + X dX^T and dA =
 * sum dS^ S~ + S^ dS~ (Sec. 3.2, Sec. 4.2.4); of the kept eigenvectors,
 * du_k = sum over discarded l of v_l (v_l . dA u_k) / (lambda_k - lambda_l)
 * (Sec. 4.2.5; rotations inside the kept space are a change of basis on a
 * bond whose two ends share the isometry, so ln Z does not depend on them);
 * of the new tensor by the product rule over its two copies of T and its
 * 2(d-1) isometries (Sec. 4.2.9); and of the trace bookkeeping (Secs. 4.1.1,
 * 4.2.16).  Pairs with |lambda_k - lambda_l| <= 1e-12 lambda_1 across the
 * cut (1e-8 lambda_1 when the step's contraction is split BF16, whose rounding
 * splits exact degeneracies by about that much) have no derivative: their
 * terms are left out, and counted when their coupling |v_l . dA u_k| exceeds
 * 1e-9 lambda_1.  While on, the contraction
 * runs densely (not in Z2 blocks; the Grams and the eigen-solver keep the
 * block form of hotrg_set_z2, whose eigenvectors have exact parities) in the
 * arithmetic of hotrg_set_precision: FP64, or split BF16 on the tensor cores
 * with the derivative's FP32 chain operands and an FP64 sum of dB before it
 * is split.  A step costs about three dense forward steps; hotrg_step waits
 * once per step for the isometry choice.
 * enable = 1 needs a context from hotrg_init_ising with beta > 0 and no step
 * yet (dT^(0) is the beta-derivative of Eq. 2.4); enable = 0 stops carrying
 * it.  hotrg_set_tensor turns it off.
 * enable = 2 carries d2T = d^2 T / d beta^2 as well, in the FP64 form only
 * (precision HOTRG_PREC_FP64, which then cannot be changed), with dense Grams
 * and eigen-solver: every bilinear stage adds f(d2X, Y) + 2 f(dX, dY) +
 * f(X, d2Y), and the kept isometry its second derivative in the parallel-
 * transport gauge, d2U = P'' U + P' P' U, P' and P'' the derivatives of the
 * projector on the kept eigenvectors (in the eigenbasis: divided differences
 * of the kept-set indicator times V^T dA V and V^T d2A V; terms across a
 * degenerate cut left out as in the first order).  hotrg_specific_heat then
 * returns d^2(ln Z/V)/d beta^2.  A step costs about twice a step carrying
 * the first derivative only (3D chi = 12: 7.4 s against 3.7 s).  Errors: EINVAL (not an Ising context, beta = 0, steps already
 * taken, enable = 2 with a split precision), ENOMEM, ECUDA, ESTATE. */
int hotrg_set_tangent(hotrg_ctx* ctx, int enable);

/* After synchronising: *d2lnz_dbeta2 = d^2(ln Z^(p) / 2^p)/d beta^2 of the
 * last step and *specific_heat = beta^2 times it (the specific heat per site).
 * Any out-pointer may be NULL.  Errors: EINVAL, ESTATE (second order not
 * carried: hotrg_set_tangent(ctx, 2)), a recorded device failure. */
int hotrg_specific_heat(hotrg_ctx* ctx, double* d2lnz_dbeta2, double* specific_heat);

/* After synchronising: *dlnz_dbeta = d(ln Z^(p) / 2^p)/d beta of the last
 * step (of T^(0) before any step), *energy = its negative (the internal
 * energy per site, bond and field terms), *degenerate_pairs = eigen pairs
 * left out so far (see hotrg_set_tangent).  Any out-pointer may be NULL.
 * Errors: EINVAL, ESTATE (derivative not carried), a recorded device failure. */
int hotrg_energy(hotrg_ctx* ctx, double* dlnz_dbeta, double* energy, int* degenerate_pairs);

/* dT/d beta of the current normalised tensor, d(T / Tr T), in the layout of
 * hotrg_tensor.  Errors: as hotrg_tensor, and ESTATE if not carried. */
int hotrg_tangent_tensor(hotrg_ctx* ctx, double* dT, int64_t cap, int dims[8]);

/* The isometry U~ chosen by the last step for lattice axis `leg` (a
 * transverse axis of that step): a rows x cols row-major FP64 matrix, rows
 * = chi_leg^2 indexed by (hat + check * chi_leg) (Sec. 3.2), cols =
 * chi_leg^new; *chosen_prime = 1 if U'^(j) (prime side) was chosen, else 0
 * (Sec. 4.2.7).  Each column is sign-fixed: its pivot entry (the lowest row
 * whose magnitude is within 1e-6 of the column's largest) is positive.
 * cap is the capacity of U in elements.  Errors: EINVAL (leg not transverse
 * in the last step, cap too small), ESTATE, a recorded device failure. */
int hotrg_isometry(hotrg_ctx* ctx, int leg, double* U, int64_t cap, int* rows,
                   int* cols, int* chosen_prime);

/* Eigenvalues, descending, of A^(j) (prime = 0) or A'^(j) (prime = 1) for
 * lattice axis `leg` in the last step (Sec. 4.2.5); *n = chi_leg^2. */
int hotrg_spectrum(hotrg_ctx* ctx, int leg, int prime, double* lam, int64_t cap, int* n);

/* FP64 one-sided Jacobi sweeps used for lattice axis `leg` in the last step. */
int hotrg_jacobi_sweeps(hotrg_ctx* ctx, int leg, int* sweeps);

/* Discarded sums epsilon^(j), epsilon'^(j) of the last step (Sec. 2). */
int hotrg_truncation(hotrg_ctx* ctx, int leg, double* eps, double* eps_prime);

/* ln Z^(p) / V^(p) with V^(p) = 2^p (Sec. 4.1.1, Eqs. eq_lnZ, K_recurrence)
 * after p steps, and f = -(ln Z/V) / beta (NaN when beta = 0). */
int hotrg_free_energy(hotrg_ctx* ctx, double* lnZ_per_site, double* f_per_site);

/* Tr T^(p) of the last new tensor before normalisation (= trace Y), the
 * Gu-Wen ratio X = (trace Y)^2 / trace(Y^2) (Sec. 4.1.2), and p. */
int hotrg_observables(hotrg_ctx* ctx, double* trace, double* gu_wen_X, int* nsteps);

/* Current bond dimension of each lattice axis (dims[k], k < d). */
int hotrg_bond_dims(hotrg_ctx* ctx, int dims[4]);

/* Copy the current normalised local tensor in interchange layout.  dims
 * receives the 2d extents.  Errors: EINVAL if cap is too small. */
int hotrg_tensor(hotrg_ctx* ctx, double* T, int64_t cap, int dims[8]);

/* The bottleneck contraction of Eq. (BottleneckPart) on its own:
 * C[M][N] = sum_k A[M][K] B[N][K] (both operands K-contiguous, row-major,
 * FP64 in and out) computed with the kernels of precision `mode` (split-BF16
 * or split-TF32 pieces on the tensor cores with FP32 accumulation, or FP64
 * DFMA tiles).
 * A, B, C may be host or device pointers.  Synchronous; allocates and frees
 * its own device scratch.  1 <= M, N, K <= 2^20 and M*K, N*K, M*N <= 2^31.
 * Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT. */
int hotrg_gemm_nt(int mode, int M, int N, int K, const double* A, const double* B, double* C);

/* hotrg_gemm_nt without any device allocation (the paper has no counterpart;
 * this serves callers that cannot allocate).  Some callers may not call
 * cudaMalloc or cudaFree: code running inside a framework that owns all
 * device memory through its own pool (a raw allocation bypasses the pool and
 * can fail once the pool has reserved the memory), and latency-critical
 * loops where cudaMalloc/cudaFree would synchronise the device.  This entry
 * point computes C[M][N] = sum_k A[M][K] B[N][K] like hotrg_gemm_nt, but A, B
 * and C must be DEVICE pointers (FP64, row-major) owned by the caller, and all
 * scratch (BF16 pieces, FP32 product, error word) lives in one fixed
 * file-scope device array of HOTRG_NOALLOC_SCRATCH_BYTES (64 MiB) that every
 * GPU loading the library keeps until the process exits.  In the BF16 modes
 * the scratch is 256 + r(2*np*M*Kp) + r(2*np*N*Kp) + r(4*M*N) bytes, with
 * np = 2 (BF16X3) or 3 (BF16X6), Kp = K rounded up to a multiple of 64 and
 * r(x) = x rounded up to a multiple of 256; sizes whose scratch exceeds the
 * array are rejected with HOTRG_EINVAL (the FP64 mode needs no scratch).
 * mode is HOTRG_PREC_FP64, HOTRG_PREC_BF16X3 or HOTRG_PREC_BF16X6 (the TF32
 * modes give HOTRG_EINVAL here).  The
 * size limits of hotrg_gemm_nt apply in every mode.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  Work is enqueued on
 * `stream` (a cudaStream_t, NULL = legacy default stream) and the call
 * returns after synchronising it.  Every call shares the one array: calls
 * that overlap on the GPU (other streams, other threads) race and must not
 * be issued.  It calls no cudaMalloc, cudaFree or allocating library routine.
 * Errors: EINVAL, ECUDA, ETIMEOUT. */
#define HOTRG_NOALLOC_SCRATCH_BYTES (64u << 20)
int hotrg_gemm_nt_noalloc(int mode, int M, int N, int K, const double* A, const double* B,
                          double* C, void* stream);

/* Rate probe of the bottleneck GEMM kernel alone: allocates operand pieces of
 * an M x K and an N x K operand (values exact in BF16 and TF32) and an FP32
 * product on the current device, launches the split tensor-core GEMM of
 * hotrg_gemm_nt once to warm up, then `iters` times back to back on the legacy
 * default stream, and returns the mean milliseconds per launch (CUDA events).
 * For rooflines and tuning; the paper has no counterpart.  mode is any split
 * mode (BF16X3, BF16X6, TF32, TF32X3).  Errors: EINVAL, ENOMEM, ECUDA,
 * ETIMEOUT. */
int hotrg_gemm_rate(int mode, int M, int N, int K, int iters, double* ms_per_launch);

/* FP64 fused multiply-add rate of the current device, in TFLOP/s (2 flops per
 * FMA): independent FMA chains on every SM, timed with CUDA events (best of
 * two launches after one warm-up).  The denominator of the FP64 kernels'
 * roofline (environment Grams, eigen-solver, the FP64 form of the
 * contraction); the paper has no counterpart.  Synchronous on the legacy
 * default stream; allocates 8 bytes per CTA for its outputs.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int hotrg_fp64_rate(double* tflops);

/* Bytes of device memory the context holds now. */
int hotrg_device_bytes(hotrg_ctx* ctx, size_t* bytes);

/* Number of kernels the context has launched since it was created. */
int hotrg_launch_count(hotrg_ctx* ctx, int64_t* launches);

void hotrg_free(hotrg_ctx* ctx);
const char* hotrg_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* HOTRG_H */
