"""Plain FP64 CPU oracle for the beta-derivative of a HOTRG run (internal energy).

TEST INFRASTRUCTURE ONLY, like ``hotrg_oracle``: nothing in the product path may
import, call or execute this module.  It builds on the forward oracle in
``hotrg_oracle`` and shares no code with the CUDA library.

The quantity is u = -d(ln Z / V)/d beta of the HOTRG approximation itself: the
run of Secs. 4.1-4.2 is differentiated step by step in forward mode, every
tensor T carrying its derivative dT = dT/d beta alongside.

  * dT^(0)/d beta of Eq. (2.4) by the product rule ........................ Sec. 2
  * d of the environments: dS = dX X^T + X dX^T, dA = sum dS^ S~ + S^ dS~ ... Sec. 3.2; Sec. 4.2.4
  * d of the kept eigenvectors of A (first-order perturbation) ........... Sec. 4.2.5
  * d of the new tensor: product rule over its two copies of T and its
    2(d-1) isometries ...................................................... Sec. 4.2.9
  * d ln Tr, d of the normalisation and of the K recurrence ............... Secs. 4.1.1, 4.2.16

Readings (the paper does not differentiate HOTRG; these are the standard
first-order results, written out here):
  * eigenvector derivative: for a kept eigenvector u_k of the symmetric A,
    du_k = sum over DISCARDED l of v_l (v_l . dA u_k) / (lambda_k - lambda_l).
    The terms with l kept rotate the kept basis among itself; such a rotation
    is an orthogonal change of basis on a bond and both ends of that bond carry
    the same isometry, so it leaves ln Z unchanged and is left out.
  * pairs (k kept, l discarded) with |lambda_k - lambda_l| <= 1e-12 lambda_1
    have no derivative (the truncation is not differentiable there); their terms
    are left out, and counted when their coupling |v_l . dA u_k| exceeds
    1e-9 lambda_1 (a pair kept apart by a symmetry of dA, such as opposite Z2
    parity, has zero coupling and is harmless).
  * the choice between U and U' (epsilon vs epsilon') and the sign gauge are
    locally constant in beta and contribute nothing.
  * beta > 0: dX_{s1}/d beta = sigma cosh / (2 sqrt(sinh)) is infinite at beta = 0.
"""

from __future__ import annotations

import math
import string
from dataclasses import dataclass

import numpy as np

from oracle import hotrg_oracle as o

DEGENERATE_REL = 1e-12


def initial_tensor_dbeta(d: int, beta: float, h: float) -> np.ndarray:
    """dT/d beta of T = sum_s V_s X_{s j1} .. X_{s jd'} (Eq. 2.4), by the product rule.

    X_{s0} = sqrt(cosh b), X_{s1} = sigma_s sqrt(sinh b), V_s = exp(b h sigma_s):
    dX_{s0} = sinh b / (2 sqrt(cosh b)), dX_{s1} = sigma_s cosh b / (2 sqrt(sinh b)),
    dV_s = h sigma_s V_s.
    """
    if not beta > 0.0:
        raise ValueError("the derivative of sqrt(sinh beta) needs beta > 0")
    x = o.ising_factor_matrix(beta)
    sigma = np.array([1.0, -1.0])
    dx = np.empty((2, 2))
    dx[:, 0] = math.sinh(beta) / (2.0 * math.sqrt(math.cosh(beta)))
    dx[:, 1] = sigma * math.cosh(beta) / (2.0 * math.sqrt(math.sinh(beta)))
    v = o.ising_site_weights(beta, h)
    dv = h * sigma * v
    nleg = 2 * d
    dt = np.zeros((2,) * nleg)
    for s in range(2):
        # d of V_s prod_legs X: one term per factor that is differentiated
        for which in range(-1, nleg):
            term = np.array(dv[s] if which < 0 else v[s])
            for leg in range(nleg):
                term = np.multiply.outer(term, dx[s] if leg == which else x[s])
            dt += term
    return dt


# ----------------------------------------------------------------------------
# Sec. 3.2 / 4.2.4: derivative of the environments
# ----------------------------------------------------------------------------

def _gram_dot(tp: np.ndarray, dtp: np.ndarray, keep: list[int]) -> np.ndarray:
    """d/d beta of G = sum over the axes not in keep of T[..k..] T[..l..]."""
    rest = [ax for ax in range(tp.ndim) if ax not in keep]
    return np.tensordot(dtp, tp, axes=(rest, rest)) + np.tensordot(tp, dtp, axes=(rest, rest))


def environment_matrix_dot(tp: np.ndarray, dtp: np.ndarray, j: int, prime: bool) -> np.ndarray:
    """dA^(j) (or dA'^(j)): the derivative of A = sum_{rho eta} S^ S~ with the same
    index conventions as ``hotrg_oracle.environment_matrix``."""
    d = tp.ndim // 2
    pj = o._pos_np(d, j) if prime else o._pos_n(d, j)
    pc, pcp = 2 * d - 2, 2 * d - 1
    s_hat = np.transpose(o._gram(tp, [pj, pcp]), (0, 2, 1, 3))
    s_check = np.transpose(o._gram(tp, [pj, pc]), (0, 2, 1, 3))
    ds_hat = np.transpose(_gram_dot(tp, dtp, [pj, pcp]), (0, 2, 1, 3))
    ds_check = np.transpose(_gram_dot(tp, dtp, [pj, pc]), (0, 2, 1, 3))
    chi = tp.shape[pj]
    a4 = np.einsum("abre,fgre->fagb", ds_hat, s_check) + np.einsum("abre,fgre->fagb", s_hat, ds_check)
    a = a4.reshape(chi * chi, chi * chi)
    return 0.5 * (a + a.T)


# ----------------------------------------------------------------------------
# Sec. 4.2.5: derivative of the kept eigenvectors
# ----------------------------------------------------------------------------

def kept_eigenvector_dot(lam: np.ndarray, v: np.ndarray, chi_new: int, da: np.ndarray):
    """du_k = sum_{l >= chi_new} v_l (v_l . dA u_k) / (lam_k - lam_l) for the
    sorted, gauged eigenpairs (lam, v) of A; returns (dU, number of degenerate
    pairs left out)."""
    n = v.shape[0]
    u = v[:, :chi_new]
    du = np.zeros_like(u)
    tol = DEGENERATE_REL * lam[0]
    z = v.T @ da @ u                       # z[l, k] = v_l . dA u_k
    skipped = 0
    for k in range(chi_new):
        for l in range(chi_new, n):
            gap = lam[k] - lam[l]
            if abs(gap) <= tol:
                if abs(z[l, k]) > 1e-9 * lam[0]:
                    skipped += 1
                continue
            du[:, k] += v[:, l] * (z[l, k] / gap)
    return du, skipped


# ----------------------------------------------------------------------------
# Sec. 4.2.9: the new tensor as one contraction, with separate operands
# ----------------------------------------------------------------------------

def contract_new(t_hat: np.ndarray, t_chk: np.ndarray, us_p: list[np.ndarray],
                 us_n: list[np.ndarray]) -> np.ndarray:
    """T^new_{n.. n'.. c c'} = sum T^_{n^.. n^'.. c rho} T~_{n~.. n~'.. rho c'}
    prod_j U_n^(j)_{(n^_j n~_j), n_j} U_p^(j)_{(n^'_j n~'_j), n'_j}   (Sec. 4.2.9)

    over the paper order (n_{d-1}..n_1, n'_{d-1}..n'_1, c, c'), in the order of
    Sec. 4.2.9: the primed isometries on the check copy, the bottleneck sum over
    (n^', rho) with the hat copy, then the unprimed isometries.  The hat copy
    keeps c open, the check copy c'; the combined index of U is hat + check * chi_j.
    With t_hat = t_chk and us_p = us_n this is ``hotrg_oracle.new_tensor``;
    separate operands give the terms of its derivative.
    """
    d = t_hat.ndim // 2
    letters = iter(string.ascii_letters)
    hat_n = [next(letters) for _ in range(d - 1)]      # n^_{d-1} .. n^_1 (array order)
    hat_np = [next(letters) for _ in range(d - 1)]
    chk_n = [next(letters) for _ in range(d - 1)]
    chk_np = [next(letters) for _ in range(d - 1)]
    new_n = [next(letters) for _ in range(d - 1)]
    new_np = [next(letters) for _ in range(d - 1)]
    c, cp, rho = next(letters), next(letters), next(letters)

    def u3(u, pos):   # U as [check, hat, new]: row hat + check * chi_j
        chi_j = t_hat.shape[pos]
        return u.reshape(chi_j, chi_j, -1)

    # primed isometries on the check copy: n~'_j -> (n^'_j, n'_j)
    x, sx = t_chk, chk_n + chk_np + [rho, cp]
    for j in range(1, d):
        pos = d - 1 - j                       # array position of n_j among the d-1
        out = [l for l in sx if l != chk_np[pos]] + [hat_np[pos], new_np[pos]]
        x = np.einsum("".join(sx) + "," + chk_np[pos] + hat_np[pos] + new_np[pos] + "->" + "".join(out),
                      x, u3(us_p[j - 1], pos), optimize=True)
        sx = out
    # bottleneck: sum over (n^', rho) with the hat copy
    sh = hat_n + hat_np + [c, rho]
    out = hat_n + [c] + [l for l in sx if l not in hat_np and l != rho]
    x = np.einsum("".join(sh) + "," + "".join(sx) + "->" + "".join(out), t_hat, x, optimize=True)
    sx = out
    # unprimed isometries: (n^_j, n~_j) -> n_j
    for j in range(d - 1, 0, -1):
        pos = d - 1 - j
        out = [l for l in sx if l not in (chk_n[pos], hat_n[pos])] + [new_n[pos]]
        x = np.einsum("".join(sx) + "," + chk_n[pos] + hat_n[pos] + new_n[pos] + "->" + "".join(out),
                      x, u3(us_n[j - 1], pos), optimize=True)
        sx = out
    final = new_n + new_np + [c, cp]
    return np.einsum("".join(sx) + "->" + "".join(final), x)


def new_tensor_dot(tp: np.ndarray, dtp: np.ndarray, us: list[np.ndarray],
                   dus: list[np.ndarray]) -> np.ndarray:
    """dT^new: the product rule over the two copies of T and the 2(d-1) isometries."""
    d = tp.ndim // 2
    out = contract_new(dtp, tp, us, us) + contract_new(tp, dtp, us, us)
    for j in range(1, d):
        swapped = list(us)
        swapped[j - 1] = dus[j - 1]
        out += contract_new(tp, tp, swapped, us)      # the isometry on the primed legs n'_j
        out += contract_new(tp, tp, us, swapped)      # the isometry on the legs n_j
    return out


# ----------------------------------------------------------------------------
# One step and the run (Secs. 4.1.1, 4.2.16) with their derivatives
# ----------------------------------------------------------------------------

@dataclass
class TangentRecord:
    step: int
    ln_z_per_site: float
    dln_z_per_site: float        # d(ln Z / V)/d beta
    energy_per_site: float       # -d(ln Z / V)/d beta
    degenerate_pairs: int


def coarse_grain_tangent(t: np.ndarray, dt: np.ndarray, axis: int, chi: int, drop_du: bool = False):
    """(T_new, dT_new, legs, degenerate pairs) for one coarse-graining of the
    normalised (t, dt) along `axis`; drop_du leaves the isometry derivatives out
    (used by a test only, to show that they matter)."""
    d = t.ndim // 2
    tp = o.to_paper_order(t, axis)
    dtp = o.to_paper_order(dt, axis)
    nxt = o.next_axes(d, axis)
    legs = [o.choose_isometry(tp, j, chi, nxt[j - 1]) for j in range(1, d)]
    us = [leg.u for leg in legs]
    dus = []
    skipped = 0
    for j, leg in enumerate(legs, start=1):
        a = o.environment_matrix(tp, j, prime=leg.chose_prime)
        da = environment_matrix_dot(tp, dtp, j, prime=leg.chose_prime)
        lam, v, _ = o.sorted_eigenpairs(a)
        chi_new = leg.u.shape[1]
        if not np.array_equal(v[:, :chi_new], leg.u):
            raise AssertionError("eigen-decomposition is not reproducible")
        du, sk = kept_eigenvector_dot(lam, v, chi_new, da)
        skipped += sk
        dus.append(np.zeros_like(du) if drop_du else du)
    tnew = contract_new(tp, tp, us, us)
    dtnew = new_tensor_dot(tp, dtp, us, dus)
    return o.from_paper_order(tnew, axis), o.from_paper_order(dtnew, axis), legs, skipped


class HotrgTangentRun:
    """The run of ``hotrg_oracle.HotrgRun`` for the Ising model with d/d beta carried along.

    ln Z^(0) = ln Tr T^(0); K^(p) = 2 (K^(p-1) + ln Tr T^(p-1)); ln Z^(p) = K^(p) + ln Tr T^(p);
    T is normalised by its trace before every step.  Derivatives: d ln Tr = Tr dT / Tr T and
    d(T / Tr T) = dT / Tr T - (d ln Tr) T / Tr T.
    """

    def __init__(self, d: int, beta: float, h: float, drop_du: bool = False):
        self.d = d
        self.beta = beta
        self.drop_du = drop_du
        t = o.initial_tensor(d, beta, h)
        dt = initial_tensor_dbeta(d, beta, h)
        self.p = 0
        tr = o.trace_physical(t)
        dln_tr = o.trace_physical(dt) / tr
        self.k, self.dk = 0.0, 0.0
        self.ln_tr, self.dln_tr = math.log(tr), dln_tr
        self.ln_z, self.dln_z = self.ln_tr, dln_tr
        self.t = t / tr
        self.dt = dt / tr - dln_tr * self.t
        self.records: list[TangentRecord] = []

    def step(self, axis: int, chi: int) -> TangentRecord:
        self.k = 2.0 * (self.k + self.ln_tr)                 # Eq. K_recurrence
        self.dk = 2.0 * (self.dk + self.dln_tr)
        tnew, dtnew, _, skipped = coarse_grain_tangent(self.t, self.dt, axis, chi, self.drop_du)
        self.p += 1
        tr = o.trace_physical(tnew)
        if not (tr > 0.0 and math.isfinite(tr)):
            raise FloatingPointError(f"non-positive or non-finite trace {tr}")
        self.ln_tr = math.log(tr)
        self.dln_tr = o.trace_physical(dtnew) / tr
        self.ln_z = self.k + self.ln_tr                       # Eq. eq_lnZ
        self.dln_z = self.dk + self.dln_tr
        self.t = tnew / tr
        self.dt = dtnew / tr - self.dln_tr * self.t
        v = 2.0 ** self.p
        rec = TangentRecord(self.p, self.ln_z / v, self.dln_z / v, -self.dln_z / v, skipped)
        self.records.append(rec)
        return rec


def run_tangent(d: int, beta: float, h: float, chi: int, axes) -> list[TangentRecord]:
    r = HotrgTangentRun(d, beta, h)
    for a in axes:
        r.step(a, chi)
    return r.records
