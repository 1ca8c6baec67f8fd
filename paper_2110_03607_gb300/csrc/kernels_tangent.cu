// Forward-mode derivative of a HOTRG run with respect to beta (the internal energy
// u = -d(ln Z / V)/d beta).  Each step carries T and dT = dT/d beta; these kernels are
// the pieces that the derivative adds to the step (the contractions reuse the step's
// own kernels with dT or dU in place of T or U).
#include "hotrg_internal.cuh"
#include "../../include/hotrg.h"

namespace hotrg {

static unsigned tgrid(long long total) {
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}

// dT0/d beta of the Ising initial tensor of Sec. 2, Eq. (2.4):
// T0[e] = sum_sigma exp(beta h sigma) prod_legs x_{bit}(sigma), x_0 = sqrt(cosh beta),
// x_1 = sigma sqrt(sinh beta); d x_0 = sinh / (2 x_0), d x_1 = sigma cosh / (2 sqrt(sinh)).
__global__ void init_ising_dbeta_kernel(double* dT, int d, double beta, double h) {
  const int n = 1 << (2 * d);
  const double c = cosh(beta), sh = sinh(beta);
  const double x0 = sqrt(c), x1 = sqrt(sh);
  const double dx0 = sh / (2.0 * x0), dx1 = c / (2.0 * x1);
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < 2; ++s) {
      const double sigma = s == 0 ? 1.0 : -1.0;
      const double bw = exp(beta * h * sigma);
      double prod = 1.0, dprod = 0.0;   // product over the legs and its derivative
      for (int leg = 0; leg < 2 * d; ++leg) {
        const int bit = (e >> leg) & 1;
        const double x = bit ? sigma * x1 : x0;
        const double dx = bit ? sigma * dx1 : dx0;
        dprod = dprod * x + prod * dx;
        prod *= x;
      }
      acc += bw * (h * sigma * prod + dprod);
    }
    dT[e] = acc;
  }
}

void launch_init_ising_dbeta(double* dT, int d, double beta, double h, cudaStream_t s) {
  init_ising_dbeta_kernel<<<1, 256, 0, s>>>(dT, d, beta, h);
  ++g_launches;
}

// dS[i][j] = sum_z (P_z[i][j] + P_z[j][i]): the derivative of a Gram X X^T from the
// split-K partials of P = dX X^T
__global__ void sym_sum_kernel(const double* __restrict__ parts, int nsplit, int m, double* __restrict__ dS) {
  const long long total = (long long)m * m;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    double acc = 0.0;
    for (int z = 0; z < nsplit; ++z)
      acc += parts[z * total + (long long)i * m + j] + parts[z * total + (long long)j * m + i];
    dS[e] = acc;
  }
}

void launch_sym_sum(const double* parts, int nsplit, int m, double* dS, cudaStream_t s) {
  sym_sum_kernel<<<tgrid((long long)m * m), 256, 0, s>>>(parts, nsplit, m, dS);
  ++g_launches;
}

// dA = sum_{rho eta} (dS^ S~ + S^ dS~), the derivative of the A of Sec. 3.2 (same index
// conventions as the step's assembly)
__global__ void assemble_dot_kernel(const double* __restrict__ sh, const double* __restrict__ dsh,
                                    const double* __restrict__ sc, const double* __restrict__ dsc,
                                    int chi, int chc, double* __restrict__ dA) {
  const int n = chi * chi, m = chi * chc;
  const long long total = (long long)n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i > j) continue;
    const int fh = i % chi, fc = i / chi, gh = j % chi, gc = j / chi;
    const long long oh = (long long)(fh * chc) * m + gh * chc, oc = (long long)(fc * chc) * m + gc * chc;
    double acc = 0.0;
    for (int rho = 0; rho < chc; ++rho)
      for (int eta = 0; eta < chc; ++eta) {
        const long long k = (long long)rho * m + eta;
        acc = fma(dsh[oh + k], sc[oc + k], acc);
        acc = fma(sh[oh + k], dsc[oc + k], acc);
      }
    dA[(long long)i * n + j] = acc;
    dA[(long long)j * n + i] = acc;
  }
}

void launch_assemble_dot(const double* sh, const double* dsh, const double* sc, const double* dsc, int chi_j,
                         int chi_c, double* dA, cudaStream_t s) {
  assemble_dot_kernel<<<tgrid((long long)chi_j * chi_j * chi_j * chi_j), 256, 0, s>>>(sh, dsh, sc, dsc, chi_j,
                                                                                     chi_c, dA);
  ++g_launches;
}

// First-order change of the kept eigenvectors (eigen-decomposition of Sec. 4.2.5):
// du_k = sum over discarded l of v_l (v_l . dA u_k) / (lam_k - lam_l).  Input
// Z[i][k] = v_i . dA u_k over the unsorted eigenvectors i, whose rank in the sorted
// order is rank[i]; output Zt[k][i] = Z[i][k] / (lam_k - lam_i) for discarded i, else 0.
// Pairs closer than rel_tol lam_1 have no derivative: left out, and counted unless their
// coupling |Z| is below 1e-9 lam_1 (a pair kept apart by a symmetry of dA, e.g. of
// opposite Z2 parity, couples with Z = 0).  rel_tol is 1e-12 with an FP64 contraction
// and 1e-8 with the split-BF16 one, whose rounding (not symmetric under the lattice
// symmetries) splits exactly degenerate pairs by about that much.
__global__ void eig_dscale_kernel(const double* __restrict__ Z, const double* __restrict__ lam_sorted,
                                  const int* __restrict__ rank, int n, int nnew, double rel_tol,
                                  double* __restrict__ Zt, TanState* tst) {
  const double tol = rel_tol * lam_sorted[0];
  const int total = n * nnew;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int k = e / n, i = e % n;
    const int ri = rank[i];
    double v = 0.0;
    if (ri >= nnew) {
      const double den = lam_sorted[k] - lam_sorted[ri];
      const double z = Z[(long long)i * nnew + k];
      if (fabs(den) > tol) v = z / den;
      else if (fabs(z) > 1e-9 * lam_sorted[0]) atomicAdd(&tst->degenerate, 1);
    }
    Zt[(long long)k * n + i] = v;
  }
}

void launch_eig_dscale(const double* Z, const double* lam_sorted, const int* rank, int n, int nnew,
                       double rel_tol, double* Zt, TanState* tst, cudaStream_t s) {
  eig_dscale_kernel<<<tgrid((long long)n * nnew), 256, 0, s>>>(Z, lam_sorted, rank, n, nnew, rel_tol, Zt, tst);
  ++g_launches;
}

// out[c][r] = in[r][c] for an rows x cols row-major matrix
__global__ void transpose_kernel(const double* __restrict__ in, int rows, int cols, double* __restrict__ out) {
  const long long total = (long long)rows * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e % cols);
    out[(long long)c * rows + r] = in[e];
  }
}

void launch_transpose(const double* in, int rows, int cols, double* out, cudaStream_t s) {
  transpose_kernel<<<tgrid((long long)rows * cols), 256, 0, s>>>(in, rows, cols, out);
  ++g_launches;
}

// y[i] = a x[i] + b y[i]
__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, double* __restrict__ y,
                             long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

void launch_axpby(double a, const double* x, double b, double* y, long long n, cudaStream_t s) {
  axpby_kernel<<<tgrid(n), 256, 0, s>>>(a, x, b, y, n);
  ++g_launches;
}

// y[i] += x[i] (FP32 chain operands of the split-BF16 form)
__global__ void add_f32_kernel(const float* __restrict__ x, float* __restrict__ y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += x[i];
}

void launch_add_f32(const float* x, float* y, long long n, cudaStream_t s) {
  add_f32_kernel<<<tgrid(n), 256, 0, s>>>(x, y, n);
  ++g_launches;
}

// out[i] = (float)in[i]
__global__ void narrow_f64_kernel(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

void launch_narrow_f64(const double* in, float* out, long long n, cudaStream_t s) {
  narrow_f64_kernel<<<tgrid(n), 256, 0, s>>>(in, out, n);
  ++g_launches;
}

// d of the trace bookkeeping of finish_step (Secs. 4.1.1, 4.2.16), after it has run:
//   d ln Tr_p = Tr dT^(p) / Tr T^(p),
//   d kappa_p = d kappa_{p-1} + d ln Tr_{p-1} / 2^(p-1),  d(ln Z^(p)/V) = d kappa_p + d ln Tr_p / 2^p
// (first: d ln Z^(0) = d ln Tr T^(0)).  Yd is the Y matrix of dT^(p).
__global__ void finish_tangent_kernel(const double* __restrict__ Yd, int chi_c, const DevState* st, TanState* tst,
                                      int p, int first) {
  if (threadIdx.x != 0) return;
  double dtr = 0.0;
  for (int c = 0; c < chi_c; ++c) dtr += Yd[c * chi_c + c];
  const double dln_tr = dtr / st->trace;
  if (first) {
    tst->dkappa = 0.0;
    tst->dln_z_site = dln_tr;
  } else {
    tst->dkappa = tst->dkappa + ldexp(tst->dln_tr, -(p - 1));
    tst->dln_z_site = tst->dkappa + ldexp(dln_tr, -p);
  }
  tst->dln_tr = dln_tr;
  tst->dtrace = dtr;
}

void launch_finish_tangent(const double* Yd, int chi_c, const DevState* st, TanState* tst, int p, int first,
                           cudaStream_t s) {
  finish_tangent_kernel<<<1, 32, 0, s>>>(Yd, chi_c, st, tst, p, first);
  ++g_launches;
}

// d(T / Tr T) = dT / Tr T - (d ln Tr) (T / Tr T): out = dT * inv_trace - dln_tr * That
__global__ void tangent_scale_kernel(const double* __restrict__ dT, const double* __restrict__ That,
                                     double* __restrict__ out, long long n, const DevState* st,
                                     const TanState* tst) {
  const double f = st->inv_trace, g = tst->dln_tr;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = dT[i] * f - g * That[i];
}

void launch_tangent_scale(const double* dT, const double* That, double* out, long long n, const DevState* st,
                          const TanState* tst, cudaStream_t s) {
  tangent_scale_kernel<<<tgrid(n), 256, 0, s>>>(dT, That, out, n, st, tst);
  ++g_launches;
}

// ---------------------------------------------------------------------------
// Second derivative d^2 / d beta^2 (specific heat), carried beside T and dT
// ---------------------------------------------------------------------------

// d^2 T0 / d beta^2 of Eq. (2.4): per sigma the product over the field factor
// V = exp(beta h sigma) and the 2d legs, differentiated twice by the product rule
// (P'' <- P'' g + 2 P' g' + P g'' for each factor g); x_0 = sqrt(cosh), x_1 = sigma
// sqrt(sinh), x_0'' = sqrt(cosh) / 2 - sinh^2 / (4 cosh^{3/2}), x_1'' = sigma (sqrt(sinh) / 2 -
// cosh^2 / (4 sinh^{3/2})), V'' = h^2 V.
__global__ void init_ising_d2beta_kernel(double* d2T, int d, double beta, double h) {
  const int n = 1 << (2 * d);
  const double c = cosh(beta), sh = sinh(beta);
  const double x0 = sqrt(c), x1 = sqrt(sh);
  const double dx0 = sh / (2.0 * x0), dx1 = c / (2.0 * x1);
  const double ddx0 = 0.5 * x0 - sh * sh / (4.0 * c * x0), ddx1 = 0.5 * x1 - c * c / (4.0 * sh * x1);
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < 2; ++s) {
      const double sigma = s == 0 ? 1.0 : -1.0;
      const double bw = exp(beta * h * sigma);
      double p0 = bw, p1 = h * sigma * bw, p2 = h * h * bw;
      for (int leg = 0; leg < 2 * d; ++leg) {
        const int bit = (e >> leg) & 1;
        const double g0 = bit ? sigma * x1 : x0, g1 = bit ? sigma * dx1 : dx0, g2 = bit ? sigma * ddx1 : ddx0;
        p2 = p2 * g0 + 2.0 * p1 * g1 + p0 * g2;
        p1 = p1 * g0 + p0 * g1;
        p0 *= g0;
      }
      acc += p2;
    }
    d2T[e] = acc;
  }
}

void launch_init_ising_d2beta(double* d2T, int d, double beta, double h, cudaStream_t s) {
  init_ising_d2beta_kernel<<<1, 256, 0, s>>>(d2T, d, beta, h);
  ++g_launches;
}

// d^2 A = sum_{rho eta} (d2S^ S~ + 2 dS^ dS~ + S^ d2S~) (Sec. 3.2 assembly, index conventions of
// assemble_dot_kernel)
__global__ void assemble_ddot_kernel(const double* __restrict__ sh, const double* __restrict__ dsh,
                                     const double* __restrict__ d2sh, const double* __restrict__ sc,
                                     const double* __restrict__ dsc, const double* __restrict__ d2sc, int chi,
                                     int chc, double* __restrict__ d2A) {
  const int n = chi * chi, m = chi * chc;
  const long long total = (long long)n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i > j) continue;
    const int fh = i % chi, fc = i / chi, gh = j % chi, gc = j / chi;
    const long long oh = (long long)(fh * chc) * m + gh * chc, oc = (long long)(fc * chc) * m + gc * chc;
    double acc = 0.0;
    for (int rho = 0; rho < chc; ++rho)
      for (int eta = 0; eta < chc; ++eta) {
        const long long k = (long long)rho * m + eta;
        acc = fma(d2sh[oh + k], sc[oc + k], acc);
        acc = fma(2.0 * dsh[oh + k], dsc[oc + k], acc);
        acc = fma(sh[oh + k], d2sc[oc + k], acc);
      }
    d2A[(long long)i * n + j] = acc;
    d2A[(long long)j * n + i] = acc;
  }
}

void launch_assemble_ddot(const double* sh, const double* dsh, const double* d2sh, const double* sc,
                          const double* dsc, const double* d2sc, int chi_j, int chi_c, double* d2A, cudaStream_t s) {
  assemble_ddot_kernel<<<tgrid((long long)chi_j * chi_j * chi_j * chi_j), 256, 0, s>>>(sh, dsh, d2sh, sc, dsc, d2sc,
                                                                                      chi_j, chi_c, d2A);
  ++g_launches;
}

// Second derivative of a kept isometry column in the parallel-transport gauge (U' = P' U,
// U'' = P'' U + P' P' U, P the projector on the kept eigenvectors of A), in the eigenbasis:
//   Z2t[k][a] = sum_b w(a, b) G1[a][b] Gs[b][k] + [a discarded] G2s[a][k] / (lam_c - lam_a)
// with c the eigenvector kept at position k, G1[a][b] = v_a . dA v_b, Gs[b][k] = v_b . dA u_k,
// G2s[a][k] = v_a . d2A u_k, and w the divided differences of the kept-set indicator
// (2 chi[a, b, c] + chi[a, b] chi[b, c]):
//   a, b kept: 0;  a kept, b not: -1 / ((lam_a - lam_b)(lam_c - lam_b));
//   a not, b kept: -2 / ((lam_b - lam_a)(lam_c - lam_a));  a, b not: 2 / ((lam_c - lam_a)(lam_c - lam_b)).
// A term whose kept-discarded gap is within rel_tol lam_1 is left out (no derivative there).
__global__ void eig_d2_kernel(const double* __restrict__ G1, const double* __restrict__ Gs,
                              const double* __restrict__ G2s, const double* __restrict__ lam_sorted,
                              const int* __restrict__ rank, int n, int nnew, double rel_tol, double* __restrict__ Z2t) {
  const double tol = rel_tol * lam_sorted[0];
  const int total = n * nnew;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int k = e / n, a = e % n;
    const double lc = lam_sorted[k];
    const int ra = rank[a];
    const bool ka = ra < nnew;
    const double la = lam_sorted[ra];
    double acc = 0.0;
    if (!ka && fabs(lc - la) > tol) acc = G2s[(long long)a * nnew + k] / (lc - la);
    for (int b = 0; b < n; ++b) {
      const int rb = rank[b];
      const bool kb = rb < nnew;
      if (ka && kb) continue;
      const double lb = lam_sorted[rb];
      double w;
      if (ka) {   // a kept, b discarded
        const double g1 = la - lb, g2 = lc - lb;
        if (fabs(g1) <= tol || fabs(g2) <= tol) continue;
        w = -1.0 / (g1 * g2);
      } else if (kb) {   // a discarded, b kept
        const double g1 = lb - la, g2 = lc - la;
        if (fabs(g1) <= tol || fabs(g2) <= tol) continue;
        w = -2.0 / (g1 * g2);
      } else {
        const double g1 = lc - la, g2 = lc - lb;
        if (fabs(g1) <= tol || fabs(g2) <= tol) continue;
        w = 2.0 / (g1 * g2);
      }
      acc = fma(w * G1[(long long)a * n + b], Gs[(long long)b * nnew + k], acc);
    }
    Z2t[(long long)k * n + a] = acc;
  }
}

void launch_eig_d2(const double* G1, const double* Gs, const double* G2s, const double* lam_sorted, const int* rank,
                   int n, int nnew, double rel_tol, double* Z2t, cudaStream_t s) {
  eig_d2_kernel<<<tgrid((long long)n * nnew), 256, 0, s>>>(G1, Gs, G2s, lam_sorted, rank, n, nnew, rel_tol, Z2t);
  ++g_launches;
}

// d^2 of the trace bookkeeping, after finish_tangent has run for the same step:
//   d2 ln Tr_p = Tr d2T^(p) / Tr T^(p) - (d ln Tr_p)^2,
//   d2 kappa_p = d2 kappa_{p-1} + d2 ln Tr_{p-1} / 2^(p-1),  d2(ln Z^(p)/V) = d2 kappa_p + d2 ln Tr_p / 2^p
__global__ void finish_tangent2_kernel(const double* __restrict__ Yd2, int chi_c, const DevState* st, TanState* tst,
                                       int p, int first) {
  if (threadIdx.x != 0) return;
  double d2tr = 0.0;
  for (int c = 0; c < chi_c; ++c) d2tr += Yd2[c * chi_c + c];
  const double l1 = tst->dln_tr;
  const double d2ln_tr = d2tr / st->trace - l1 * l1;
  if (first) {
    tst->d2kappa = 0.0;
    tst->d2ln_z_site = d2ln_tr;
  } else {
    tst->d2kappa = tst->d2kappa + ldexp(tst->d2ln_tr, -(p - 1));
    tst->d2ln_z_site = tst->d2kappa + ldexp(d2ln_tr, -p);
  }
  tst->d2ln_tr = d2ln_tr;
}

void launch_finish_tangent2(const double* Yd2, int chi_c, const DevState* st, TanState* tst, int p, int first,
                            cudaStream_t s) {
  finish_tangent2_kernel<<<1, 32, 0, s>>>(Yd2, chi_c, st, tst, p, first);
  ++g_launches;
}

// d^2 (T / Tr T) = d2T / Tr - (d ln Tr) dT / Tr - (d ln Tr) d(T / Tr) - (d2 ln Tr) (T / Tr):
// out = d2T f - l1 dT f - l1 dThat - l2 That, f = 1 / Tr
__global__ void tangent2_scale_kernel(const double* __restrict__ d2T, const double* __restrict__ dT,
                                      const double* __restrict__ dThat, const double* __restrict__ That,
                                      double* __restrict__ out, long long n, const DevState* st, const TanState* tst) {
  const double f = st->inv_trace, l1 = tst->dln_tr, l2 = tst->d2ln_tr;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = d2T[i] * f - l1 * dT[i] * f - l1 * dThat[i] - l2 * That[i];
}

void launch_tangent2_scale(const double* d2T, const double* dT, const double* dThat, const double* That, double* out,
                           long long n, const DevState* st, const TanState* tst, cudaStream_t s) {
  tangent2_scale_kernel<<<tgrid(n), 256, 0, s>>>(d2T, dT, dThat, That, out, n, st, tst);
  ++g_launches;
}

}  // namespace hotrg
