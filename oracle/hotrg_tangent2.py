"""Plain FP64 CPU oracle for the second beta-derivative of a HOTRG run (specific heat).

TEST INFRASTRUCTURE ONLY, like ``hotrg_oracle`` and ``hotrg_tangent``: nothing in the
product path may import, call or execute this module.  It builds on those two modules
and shares no code with the CUDA library.

The run of Secs. 4.1-4.2 is differentiated twice in forward mode: every tensor T
carries dT and d2T = d^2 T / d beta^2 alongside, and the K recurrence of Sec. 4.1.1
gives d^2 (ln Z / V) / d beta^2; the specific heat per site is
c = beta^2 d^2 (ln Z / V) / d beta^2.

  * d2T^(0) of Eq. (2.4): the second product rule over its 2d + 1 factors ...... Sec. 2
  * d2 of the Grams and of A: d2(X Y) = d2X Y + 2 dX dY + X d2Y .......... Sec. 3.2; Sec. 4.2.4
  * d2 of the kept eigenvectors ........................................... Sec. 4.2.5
  * d2 of the new tensor: the second product rule over its 2d multilinear
    operands (two copies of T, 2(d-1) isometries) .......................... Sec. 4.2.9
  * d2 ln Tr and of the normalisation and the K recurrence ............... Secs. 4.1.1, 4.2.16

Readings (the paper does not differentiate HOTRG; these are standard results written
out here):
  * the kept isometry U of a step spans the leading eigenspace of A, whose projector
    P = U U^T is a smooth function of beta away from degeneracies at the cut.  U is
    carried in the parallel-transport gauge U' = P' U (no rotation inside the kept
    space, the first-order rule of ``hotrg_tangent``), so U'' = P'' U + P' P' U.  A
    rotation inside the kept space is a change of basis on a bond that both of its
    ends see, so ln Z and its derivatives do not depend on the gauge.
  * P as a function of A is chi(A) for the indicator chi of the kept eigenvalues; its
    derivatives (Daleckii-Krein) in the eigenbasis of A, with G1 = V^T dA V and
    G2 = V^T d2A V, are  P'_ac = chi[a, c] G1_ac  and
    P''_ac = sum_b 2 chi[a, b, c] G1_ab G1_bc + chi[a, c] G2_ac,
    with the divided differences of chi:
      chi[a, c] = (chi_a - chi_c) / (lam_a - lam_c)  (0 when both are kept or both not);
      chi[a, b, c] = 0 when all three are kept or none is,
                   = 1 / ((lam_k - lam_l1)(lam_k - lam_l2))  for one kept k,
                   = -1 / ((lam_k1 - lam_l)(lam_k2 - lam_l))  for two kept k1, k2.
    Only gaps between a kept and a discarded eigenvalue appear; terms with such a gap
    within DEGENERATE_REL lambda_1 are left out (as in the first order).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from oracle import hotrg_oracle as o
from oracle import hotrg_tangent as tg

DEGENERATE_REL = tg.DEGENERATE_REL


def initial_tensor_d2beta(d: int, beta: float, h: float) -> np.ndarray:
    """d^2 T / d beta^2 of T = sum_s V_s X_{s j1} .. X_{s jd'} (Eq. 2.4): one term per
    factor differentiated twice and two per unordered pair differentiated once each.

    X_{s0} = sqrt(cosh b):            X'' = sqrt(cosh b) / 2 - sinh^2 b / (4 cosh^{3/2} b)
    X_{s1} = sigma_s sqrt(sinh b):     X'' = sigma_s (sqrt(sinh b) / 2 - cosh^2 b / (4 sinh^{3/2} b))
    V_s = exp(b h sigma_s):            V'' = h^2 V_s
    """
    if not beta > 0.0:
        raise ValueError("the derivatives of sqrt(sinh beta) need beta > 0")
    ch, sh = math.cosh(beta), math.sinh(beta)
    x = o.ising_factor_matrix(beta)
    sigma = np.array([1.0, -1.0])
    dx = np.empty((2, 2))
    dx[:, 0] = sh / (2.0 * math.sqrt(ch))
    dx[:, 1] = sigma * ch / (2.0 * math.sqrt(sh))
    ddx = np.empty((2, 2))
    ddx[:, 0] = math.sqrt(ch) / 2.0 - sh * sh / (4.0 * ch ** 1.5)
    ddx[:, 1] = sigma * (math.sqrt(sh) / 2.0 - ch * ch / (4.0 * sh ** 1.5))
    v = o.ising_site_weights(beta, h)
    dv = h * sigma * v
    ddv = h * h * v
    nleg = 2 * d
    out = np.zeros((2,) * nleg)
    # factor -1 is V_s, factors 0 .. nleg-1 the legs
    for s in range(2):
        def factor(f, order):
            if f < 0:
                return np.array((v[s], dv[s], ddv[s])[order])
            return (x[s], dx[s], ddx[s])[order]

        for f1 in range(-1, nleg):
            for f2 in range(f1, nleg):
                coef = 1.0 if f1 == f2 else 2.0
                term = np.array(factor(-1, 2 if f1 == f2 == -1 else (1 if -1 in (f1, f2) else 0)))
                for leg in range(nleg):
                    order = (leg == f1) + (leg == f2)
                    term = np.multiply.outer(term, factor(leg, order))
                out += coef * term
    return out


# ----------------------------------------------------------------------------
# Sec. 3.2 / 4.2.4: second derivative of the environments
# ----------------------------------------------------------------------------

def _gram2(x: np.ndarray, y: np.ndarray, keep: list[int]) -> np.ndarray:
    rest = [ax for ax in range(x.ndim) if ax not in keep]
    return np.tensordot(x, y, axes=(rest, rest))


def _gram_ddot(tp, dtp, ddtp, keep):
    """d^2 of G = sum over the axes not in keep of T[..k..] T[..l..]."""
    return _gram2(ddtp, tp, keep) + 2.0 * _gram2(dtp, dtp, keep) + _gram2(tp, ddtp, keep)


def environment_matrix_ddot(tp, dtp, ddtp, j: int, prime: bool) -> np.ndarray:
    """d^2 A^(j) (or A'^(j)) with the conventions of ``hotrg_oracle.environment_matrix``."""
    d = tp.ndim // 2
    pj = o._pos_np(d, j) if prime else o._pos_n(d, j)
    pc, pcp = 2 * d - 2, 2 * d - 1
    perm = (0, 2, 1, 3)
    s_hat = np.transpose(o._gram(tp, [pj, pcp]), perm)
    s_chk = np.transpose(o._gram(tp, [pj, pc]), perm)
    ds_hat = np.transpose(tg._gram_dot(tp, dtp, [pj, pcp]), perm)
    ds_chk = np.transpose(tg._gram_dot(tp, dtp, [pj, pc]), perm)
    dds_hat = np.transpose(_gram_ddot(tp, dtp, ddtp, [pj, pcp]), perm)
    dds_chk = np.transpose(_gram_ddot(tp, dtp, ddtp, [pj, pc]), perm)
    chi = tp.shape[pj]
    e = "abre,fgre->fagb"
    a4 = np.einsum(e, dds_hat, s_chk) + 2.0 * np.einsum(e, ds_hat, ds_chk) + np.einsum(e, s_hat, dds_chk)
    a = a4.reshape(chi * chi, chi * chi)
    return 0.5 * (a + a.T)


# ----------------------------------------------------------------------------
# Sec. 4.2.5: first and second derivative of the kept isometry
# ----------------------------------------------------------------------------

def kept_isometry_derivatives(lam: np.ndarray, v: np.ndarray, chi_new: int, da: np.ndarray,
                              dda: np.ndarray):
    """(dU, d2U, degenerate pairs left out) of U = the first chi_new columns of the sorted,
    gauged eigenvectors v of A, in the parallel-transport gauge: dU = P' U,
    d2U = P'' U + P' P' U with the divided-difference forms of the module docstring."""
    n = v.shape[0]
    kept = np.zeros(n, dtype=bool)
    kept[:chi_new] = True
    tol = DEGENERATE_REL * lam[0]
    g1 = v.T @ da @ v
    g2 = v.T @ dda @ v
    # chi[a, c]
    c1 = np.zeros((n, n))
    skipped = 0
    for a in range(n):
        for c in range(n):
            if kept[a] == kept[c]:
                continue
            gap = lam[a] - lam[c]
            if abs(gap) <= tol:
                if kept[c] and abs(g1[a, c]) > 1e-9 * lam[0]:
                    skipped += 1
                continue
            c1[a, c] = (float(kept[a]) - float(kept[c])) / gap

    def c2(a, b, c):
        ks = [i for i in (a, b, c) if kept[i]]
        ls = [i for i in (a, b, c) if not kept[i]]
        if len(ks) in (0, 3):
            return 0.0
        if len(ks) == 1:
            g_1, g_2 = lam[ks[0]] - lam[ls[0]], lam[ks[0]] - lam[ls[1]]
            if abs(g_1) <= tol or abs(g_2) <= tol:
                return 0.0
            return 1.0 / (g_1 * g_2)
        g_1, g_2 = lam[ks[0]] - lam[ls[0]], lam[ks[1]] - lam[ls[0]]
        if abs(g_1) <= tol or abs(g_2) <= tol:
            return 0.0
        return -1.0 / (g_1 * g_2)

    p1 = c1 * g1                                  # P' in the eigenbasis
    p2 = np.zeros((n, chi_new))                   # P'' restricted to kept columns
    for a in range(n):
        for c in range(chi_new):
            acc = 0.0
            for b in range(n):
                w = c2(a, b, c)
                if w != 0.0:
                    acc += 2.0 * w * g1[a, b] * g1[b, c]
            p2[a, c] = acc + c1[a, c] * g2[a, c]
    du = v @ p1[:, :chi_new]
    ddu = v @ (p2 + (p1 @ p1)[:, :chi_new])
    return du, ddu, skipped


# ----------------------------------------------------------------------------
# Sec. 4.2.9: second derivative of the new tensor (multilinear in 2d operands)
# ----------------------------------------------------------------------------

def new_tensor_ddot(tp, dtp, ddtp, us, dus, ddus) -> np.ndarray:
    """d^2 T^new: operands (T^, T~, U_p^(1..d-1), U_n^(1..d-1)) of ``hotrg_tangent.contract_new``,
    each twice differentiated once, each pair differentiated once each (both orders)."""
    d = tp.ndim // 2
    m = 2 * d
    vals = [(tp, dtp, ddtp), (tp, dtp, ddtp)] + [(u, du, ddu) for u, du, ddu in zip(us, dus, ddus)] * 2

    def call(orders):
        ops = [vals[i][orders[i]] for i in range(m)]
        return tg.contract_new(ops[0], ops[1], ops[2: 2 + (d - 1)], ops[2 + (d - 1):])

    out = None
    for i in range(m):
        orders = [0] * m
        orders[i] = 2
        term = call(orders)
        out = term if out is None else out + term
        for k in range(i + 1, m):
            orders = [0] * m
            orders[i] = orders[k] = 1
            out = out + 2.0 * call(orders)
    return out


def coarse_grain_tangent2(t, dt, ddt, axis: int, chi: int):
    """(T_new, dT_new, d2T_new, degenerate pairs) for one coarse-graining of the normalised
    (t, dt, ddt) along `axis`."""
    d = t.ndim // 2
    tp = o.to_paper_order(t, axis)
    dtp = o.to_paper_order(dt, axis)
    ddtp = o.to_paper_order(ddt, axis)
    nxt = o.next_axes(d, axis)
    legs = [o.choose_isometry(tp, j, chi, nxt[j - 1]) for j in range(1, d)]
    us, dus, ddus = [], [], []
    skipped = 0
    for j, leg in enumerate(legs, start=1):
        a = o.environment_matrix(tp, j, prime=leg.chose_prime)
        da = tg.environment_matrix_dot(tp, dtp, j, prime=leg.chose_prime)
        dda = environment_matrix_ddot(tp, dtp, ddtp, j, prime=leg.chose_prime)
        lam, v, _ = o.sorted_eigenpairs(a)
        chi_new = leg.u.shape[1]
        if not np.array_equal(v[:, :chi_new], leg.u):
            raise AssertionError("eigen-decomposition is not reproducible")
        du, ddu, sk = kept_isometry_derivatives(lam, v, chi_new, da, dda)
        skipped += sk
        us.append(leg.u)
        dus.append(du)
        ddus.append(ddu)
    tnew = tg.contract_new(tp, tp, us, us)
    dtnew = tg.new_tensor_dot(tp, dtp, us, dus)
    ddtnew = new_tensor_ddot(tp, dtp, ddtp, us, dus, ddus)
    return (o.from_paper_order(tnew, axis), o.from_paper_order(dtnew, axis),
            o.from_paper_order(ddtnew, axis), skipped)


@dataclass
class CurvatureRecord:
    step: int
    ln_z_per_site: float
    dln_z_per_site: float          # d(ln Z / V)/d beta
    d2ln_z_per_site: float         # d^2(ln Z / V)/d beta^2
    energy_per_site: float         # -d(ln Z / V)/d beta
    specific_heat_per_site: float  # beta^2 d^2(ln Z / V)/d beta^2
    degenerate_pairs: int


class HotrgTangent2Run:
    """The Ising run of ``hotrg_oracle.HotrgRun`` with d/d beta and d^2/d beta^2 carried.

    K^(p) = 2 (K^(p-1) + ln Tr T^(p-1)) and ln Z^(p) = K^(p) + ln Tr T^(p) are linear in the
    ln Tr, so their derivatives follow the same recurrence.  With tau = Tr T_new and
    l1 = d ln tau = tau' / tau:  d2 ln tau = tau'' / tau - l1^2, and the normalised
    T = T_new / tau has  T' = (T_new' - l1 T_new) / tau  and
    T'' = T_new'' / tau - l1 T_new' / tau - l1 T' - (d2 ln tau) T.
    """

    def __init__(self, d: int, beta: float, h: float):
        self.d = d
        self.beta = beta
        t = o.initial_tensor(d, beta, h)
        dt = tg.initial_tensor_dbeta(d, beta, h)
        ddt = initial_tensor_d2beta(d, beta, h)
        self.p = 0
        self.k = self.dk = self.ddk = 0.0
        self._normalise(t, dt, ddt)
        self.ln_z, self.dln_z, self.ddln_z = self.ln_tr, self.dln_tr, self.ddln_tr
        self.records: list[CurvatureRecord] = []

    def _normalise(self, tn, dtn, ddtn):
        tau = o.trace_physical(tn)
        if not (tau > 0.0 and math.isfinite(tau)):
            raise FloatingPointError(f"non-positive or non-finite trace {tau}")
        l1 = o.trace_physical(dtn) / tau
        l2 = o.trace_physical(ddtn) / tau - l1 * l1
        self.ln_tr, self.dln_tr, self.ddln_tr = math.log(tau), l1, l2
        self.t = tn / tau
        self.dt = dtn / tau - l1 * self.t
        self.ddt = ddtn / tau - l1 * dtn / tau - l1 * self.dt - l2 * self.t

    def step(self, axis: int, chi: int) -> CurvatureRecord:
        self.k = 2.0 * (self.k + self.ln_tr)                    # Eq. K_recurrence
        self.dk = 2.0 * (self.dk + self.dln_tr)
        self.ddk = 2.0 * (self.ddk + self.ddln_tr)
        tnew, dtnew, ddtnew, skipped = coarse_grain_tangent2(self.t, self.dt, self.ddt, axis, chi)
        self.p += 1
        self._normalise(tnew, dtnew, ddtnew)
        self.ln_z = self.k + self.ln_tr                          # Eq. eq_lnZ
        self.dln_z = self.dk + self.dln_tr
        self.ddln_z = self.ddk + self.ddln_tr
        v = 2.0 ** self.p
        rec = CurvatureRecord(self.p, self.ln_z / v, self.dln_z / v, self.ddln_z / v, -self.dln_z / v,
                              self.beta ** 2 * self.ddln_z / v, skipped)
        self.records.append(rec)
        return rec
