"""Plain FP64 CPU oracle for one HOTRG coarse-graining step and the run around it.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library and imports nothing from the package.

Method: Yamashita & Sakurai, "A Parallel Computing Method for the Higher Order
Tensor Renormalization Group" (arXiv:2110.03607), following the steps in the
paper's order and notation:

  * initial tensor from W = U Lambda U^T, X = U sqrt(Lambda) ............ Sec. 2, Eqs. (2.1)-(2.4)
  * normalisation f^(p) = 1/Tr T, trace of a local tensor ............... Sec. 3.1.3, Eq. (Trace_LocalTensor)
  * index renaming between steps ........................................ Sec. 3.1.3, Eq. (rename_indices)
  * environments S-hat, S-check and A = sum_{rho eta} S-hat S-check ...... Sec. 3.2, Eqs. (Aux_Tensor_hat_S), (Aux_Tensor_check_S); Sec. 4.2.4
  * "SVD" of the symmetric PSD A (eigenvectors, values descending) ....... Sec. 4.2.5, Eqs. (SVD_N), (SVD_P)
  * choice by the discarded sums epsilon, epsilon' ....................... Sec. 2 (criterion of Xie et al.); Secs. 4.2.6-4.2.7
  * truncation to chi_new = min(chi_j^2, chi) columns, sign gauge ........ Sec. 2; Sec. 4.2.8
  * new tensor: prime-side chain, bottleneck, non-prime chain ............ Sec. 4.2.9, Eqs. (TU1)-(TUNCD), (BottleneckPart), (AfterBNNCD)-(AfterBN1), (Elements_NewTensor)
  * Y matrix, trace and Gu-Wen ratio X ................................... Sec. 4.1.2, Eqs. (ratio_X), (Matrix_Y); Sec. 4.2.11
  * ln Z^(p) = K^(p) + ln Tr T^(p), K recurrence ......................... Sec. 4.1.1, Eqs. (eq_lnZ), (K_recurrence)

Readings where the paper is silent:
  * Ising: sigma_0 = +1, sigma_1 = -1, W_{s s'} = exp(beta s s'), V_s = exp(beta h s).
  * hat copy = the copy whose Current leg c stays open; combined index
    (hat, check) = hat + check * chi_j (Sec. 3.2, text after Eq. Contraction_NewTensor).
  * "singular values" in epsilon are the eigenvalues of A = M M^T, clamped >= 0.
  * choice: U if epsilon < epsilon' - tol, else U'; tol = 1e-10 * max(lambda_1, lambda'_1).
  * eigenvalues within 1e-12 * lambda_1 of each other are ordered by the pivot
    index of their vectors; the pivot of a vector is the lowest row whose
    magnitude is >= (1 - 1e-6) * max magnitude, and each kept column is
    flipped so that its pivot entry is positive.
  * Next j = physical axis (a + j) mod d when coarse-graining along axis a.

The eigen-solver is the cyclic two-sided Jacobi method with the round-robin
(parallel) ordering of Golub & Van Loan, "Matrix Computations", Sec. 8.5;
pairs whose off-diagonal entry is exactly zero are skipped, so an exact
block (Z2) zero pattern in A is kept exactly.

Storage convention of a local tensor here: a numpy array whose 2d axes are
(x_1, x_1', x_2, x_2', ..., x_d, x_d'), the order of Eq. (2.4); physical
axis k owns array axes 2k (unprimed) and 2k+1 (primed).
"""

from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

TIE_REL = 1e-12        # eigenvalue tie tolerance, relative to lambda_1
PIVOT_REL = 1e-6       # pivot-entry tolerance for the sign gauge
CHOICE_REL = 1e-10     # epsilon vs epsilon' tie tolerance, relative to lambda_1


# ----------------------------------------------------------------------------
# Sec. 2: model and initial tensor
# ----------------------------------------------------------------------------

def ising_factor_matrix(beta: float) -> np.ndarray:
    """X = U sqrt(Lambda) for W = U Lambda U^T, W_{s s'} = exp(beta s s') (Sec. 2).

    With sigma_0 = +1, sigma_1 = -1: U = [[1, 1], [1, -1]] / sqrt(2) and
    Lambda = diag(2 cosh beta, 2 sinh beta), so column 0 of X is even and
    column 1 is odd under the spin flip.
    """
    if beta < 0:
        raise ValueError("beta must be >= 0 (sqrt(sinh beta) is imaginary otherwise)")
    u = np.array([[1.0, 1.0], [1.0, -1.0]]) / math.sqrt(2.0)
    lam = np.array([2.0 * math.cosh(beta), 2.0 * math.sinh(beta)])
    return u * np.sqrt(lam)[None, :]


def ising_site_weights(beta: float, h: float) -> np.ndarray:
    """V_s = exp(g(sigma_s)) with g(sigma) = beta h sigma (Sec. 2, Eq. 2.2)."""
    sigma = np.array([1.0, -1.0])
    return np.exp(beta * h * sigma)


def initial_tensor(d: int, beta: float, h: float) -> np.ndarray:
    """T_{j1 j1' ... jd jd'} = sum_s X_{s j1} ... X_{s jd'} V_s (Sec. 2, Eq. 2.4).

    X is real, so X* = X.  Returned axes: (x_1, x_1', ..., x_d, x_d').
    """
    x = ising_factor_matrix(beta)
    v = ising_site_weights(beta, h)
    t = np.zeros((2,) * (2 * d))
    for s in range(2):
        term = np.array(v[s])
        for _ in range(2 * d):
            term = np.multiply.outer(term, x[s])
        t += term
    return t


# ----------------------------------------------------------------------------
# Sec. 3.1.3: trace of a local tensor; Sec. 4.1.2: Y matrix and ratio X
# ----------------------------------------------------------------------------

def trace_physical(t: np.ndarray) -> float:
    """Tr T = sum over every leg set equal to its primed partner (Eq. Trace_LocalTensor)."""
    d = t.ndim // 2
    m = t
    for _ in range(d):
        m = np.trace(m, axis1=0, axis2=1)
    return float(m)


def y_matrix_paper(tp: np.ndarray) -> np.ndarray:
    """Y_{c c'} = sum_{n~} T_{n~ ... n~ c c'} for T in the paper's order (Eq. Matrix_Y)."""
    d = tp.ndim // 2
    m = tp
    # axes: n_{d-1}..n_1 (d-1), n'_{d-1}..n'_1 (d-1), c, c'
    for k in range(d - 1):
        # pair the first remaining unprimed axis with its primed partner
        m = np.trace(m, axis1=0, axis2=d - 1 - k)
    return np.asarray(m)


def gu_wen_ratio(y: np.ndarray) -> float:
    """X = (trace Y)^2 / trace(Y^2) (Eq. ratio_X)."""
    tr = np.trace(y)
    return float(tr * tr / np.trace(y @ y))


# ----------------------------------------------------------------------------
# Sec. 4.2.5: symmetric eigen-solver (two-sided cyclic Jacobi)
# ----------------------------------------------------------------------------

def jacobi_eigh(a: np.ndarray, max_sweeps: int = 80):
    """Eigen-decomposition A = V diag(lam) V^T of a real symmetric matrix.

    Cyclic two-sided Jacobi with the round-robin ordering (Golub & Van Loan,
    Matrix Computations, Secs. 8.5.2-8.5.4): each round applies n/2 disjoint
    plane rotations, each of which zeroes one off-diagonal pair; a pair is
    rotated only if |a_pq| > eps * sqrt(|a_pp a_qq|) and |a_pq| > eps * ||A||_F
    (and never if a_pq is exactly 0).  Returns (lam, V, sweeps); lam is
    unsorted.
    """
    a = np.array(a, dtype=np.float64, copy=True)
    n = a.shape[0]
    v = np.eye(n)
    if n == 1:
        return a.diagonal().copy(), v, 0
    eps = np.finfo(np.float64).eps
    # absolute floor: off-diagonals below eps * ||A||_F are rounding noise (the
    # near-null block of a PSD matrix regenerates noise of that size with every
    # rotation against a large row) and are left alone
    floor = eps * float(np.sqrt((a * a).sum()))
    m = n + (n % 2)
    players = list(range(m))
    for sweep in range(1, max_sweeps + 1):
        rotated = False
        for _ in range(m - 1):
            pairs = [(players[i], players[m - 1 - i]) for i in range(m // 2)]
            pairs = [(min(p, q), max(p, q)) for p, q in pairs if max(p, q) < n]
            p = np.array([x for x, _ in pairs])
            q = np.array([y for _, y in pairs])
            apq = a[p, q]
            app = a[p, p]
            aqq = a[q, q]
            act = (apq != 0.0) & (np.abs(apq) > eps * np.sqrt(np.abs(app * aqq))) \
                & (np.abs(apq) > floor)
            if act.any():
                rotated = True
                p, q, apq, app, aqq = p[act], q[act], apq[act], app[act], aqq[act]
                # Golub & Van Loan sym.schur2: choose t = tan(theta) of the smaller angle
                zeta = (aqq - app) / (2.0 * apq)
                t = np.where(zeta >= 0, 1.0, -1.0) / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                # A <- A J (columns p, q), then A <- J^T A (rows p, q); V <- V J
                ap = a[:, p].copy()
                aq = a[:, q].copy()
                a[:, p] = c * ap - s * aq
                a[:, q] = s * ap + c * aq
                ap = a[p, :].copy()
                aq = a[q, :].copy()
                a[p, :] = c[:, None] * ap - s[:, None] * aq
                a[q, :] = s[:, None] * ap + c[:, None] * aq
                vp = v[:, p].copy()
                vq = v[:, q].copy()
                v[:, p] = c * vp - s * vq
                v[:, q] = s * vp + c * vq
            # round-robin rotation of the players, the first stays fixed
            players = [players[0], players[-1]] + players[1:-1]
        if not rotated:
            return a.diagonal().copy(), v, sweep
    raise RuntimeError(f"Jacobi did not converge in {max_sweeps} sweeps (n={n})")


def pivot_index(vec: np.ndarray) -> int:
    """Lowest row whose magnitude is within PIVOT_REL of the largest magnitude."""
    mag = np.abs(vec)
    top = mag.max()
    return int(np.nonzero(mag >= (1.0 - PIVOT_REL) * top)[0][0])


def sorted_eigenpairs(a: np.ndarray):
    """Eigenvalues in descending order (Sec. 4.2.5) with the tie and gauge readings.

    Negative eigenvalues of the PSD matrix A are rounding noise and are set
    to 0.  Values within TIE_REL * lambda_1 of their predecessor form a tie
    group, ordered by pivot index.  Each column is then flipped so that its
    pivot entry is positive ("we may invert it", Sec. 4.2.8).
    Returns (lam, V, sweeps).
    """
    lam, v, sweeps = jacobi_eigh(a)
    lam = np.maximum(lam, 0.0)
    order = sorted(range(len(lam)), key=lambda i: -lam[i])
    lam1 = lam[order[0]] if len(order) else 0.0
    tol = TIE_REL * lam1
    groups, cur = [], [order[0]]
    for i in order[1:]:
        if lam[cur[-1]] - lam[i] <= tol:
            cur.append(i)
        else:
            groups.append(cur)
            cur = [i]
    groups.append(cur)
    final = []
    for g in groups:
        final.extend(sorted(g, key=lambda i: pivot_index(v[:, i])))
    lam = lam[final]
    v = v[:, final].copy()
    for k in range(v.shape[1]):
        if v[pivot_index(v[:, k]), k] < 0:
            v[:, k] = -v[:, k]
    return lam, v, sweeps


# ----------------------------------------------------------------------------
# Paper index order and the environments (Secs. 3.1.3, 3.2, 4.2.4)
# ----------------------------------------------------------------------------

def next_axes(d: int, axis: int):
    """Physical axes of Next 1 .. Next d-1 when Current = axis (Sec. 3.1.2)."""
    return [(axis + j) % d for j in range(1, d)]


def to_paper_order(t: np.ndarray, axis: int) -> np.ndarray:
    """Physical layout -> T_{n_{d-1} .. n_1 n'_{d-1} .. n'_1 c c'} (Sec. 3.1.3)."""
    d = t.ndim // 2
    nxt = next_axes(d, axis)
    perm = [2 * nxt[j - 1] for j in range(d - 1, 0, -1)]
    perm += [2 * nxt[j - 1] + 1 for j in range(d - 1, 0, -1)]
    perm += [2 * axis, 2 * axis + 1]
    return np.transpose(t, perm)


def from_paper_order(tp: np.ndarray, axis: int) -> np.ndarray:
    """Inverse of to_paper_order (the renaming of Eq. rename_indices is the
    reassignment of these axes to the physical directions)."""
    d = tp.ndim // 2
    nxt = next_axes(d, axis)
    perm = [2 * nxt[j - 1] for j in range(d - 1, 0, -1)]
    perm += [2 * nxt[j - 1] + 1 for j in range(d - 1, 0, -1)]
    perm += [2 * axis, 2 * axis + 1]
    inv = np.argsort(perm)
    return np.transpose(tp, inv)


def _pos_n(d: int, j: int) -> int:
    """Array position of n_j in paper order."""
    return d - 1 - j


def _pos_np(d: int, j: int) -> int:
    """Array position of n'_j in paper order."""
    return 2 * (d - 1) - j


def _gram(tp: np.ndarray, keep: list[int]) -> np.ndarray:
    """G[k1, k2, l1, l2] = sum over every axis not in keep of T[..k..] T[..l..]."""
    rest = [ax for ax in range(tp.ndim) if ax not in keep]
    return np.tensordot(tp, tp, axes=(rest, rest))


def environment_matrix(tp: np.ndarray, j: int, prime: bool) -> np.ndarray:
    """A^(j) (prime=False) or A'^(j) (prime=True) of Sec. 3.2 / Sec. 4.2.4.

    S-hat_{f g rho eta} = sum T_{.. f .. c rho} T_{.. g .. c eta}  (sum over c and
    all legs but n_j), S-check_{f g rho eta} = sum T_{.. f .. rho c'} T_{.. g .. eta c'}
    (sum over c' and all legs but n_j), and
    A_{(f^ f~),(g^ g~)} = sum_{rho eta} S-hat_{f^ g^ rho eta} S-check_{f~ g~ rho eta}
    with (f^ f~) = f^ + f~ chi_{n_j}.  The prime side uses n'_j.
    """
    d = tp.ndim // 2
    pj = _pos_np(d, j) if prime else _pos_n(d, j)
    pc, pcp = 2 * d - 2, 2 * d - 1
    # keep (n_j, c') -> G[f, rho, g, eta]
    s_hat = np.transpose(_gram(tp, [pj, pcp]), (0, 2, 1, 3))
    # keep (n_j, c) -> G[f, rho, g, eta], rho/eta being the c index of each copy
    s_check = np.transpose(_gram(tp, [pj, pc]), (0, 2, 1, 3))
    chi = tp.shape[pj]
    # A4[f~, f^, g~, g^] so that a C-order reshape gives row f^ + f~ chi
    a4 = np.einsum("abre,fgre->fagb", s_hat, s_check)
    a = a4.reshape(chi * chi, chi * chi)
    return 0.5 * (a + a.T)


@dataclass
class LegChoice:
    """Isometry data for one transverse leg of one step."""
    axis: int                 # physical axis of the leg
    j: int                    # Next-j label in the step
    lam: np.ndarray           # eigenvalues of A^(j), descending
    lam_prime: np.ndarray     # eigenvalues of A'^(j), descending
    eps: float
    eps_prime: float
    chose_prime: bool
    u: np.ndarray             # truncated, gauged isometry (chi_j^2, chi_new)
    gap_at_cut: float
    sweeps: tuple = (0, 0)


def choose_isometry(tp: np.ndarray, j: int, chi: int, axis_phys: int) -> LegChoice:
    """U^(j) / U'^(j), epsilon, epsilon', the choice and the truncation
    (Sec. 2 criterion; Secs. 4.2.5-4.2.8)."""
    a = environment_matrix(tp, j, prime=False)
    ap = environment_matrix(tp, j, prime=True)
    lam, u, sw = sorted_eigenpairs(a)
    lamp, up, swp = sorted_eigenpairs(ap)
    n = a.shape[0]
    chi_new = min(n, chi)
    eps = float(lam[chi_new:].sum())
    epsp = float(lamp[chi_new:].sum())
    tol = CHOICE_REL * max(lam[0], lamp[0])
    chose_prime = not (eps < epsp - tol)
    lam_c, u_c = (lamp, up) if chose_prime else (lam, u)
    ut = u_c[:, :chi_new].copy()
    gap = float((lam_c[chi_new - 1] - lam_c[chi_new]) / lam_c[0]) if (chi_new < n and lam_c[0] > 0) else math.inf
    return LegChoice(axis_phys, j, lam, lamp, eps, epsp, chose_prime, ut, gap, (sw, swp))


# ----------------------------------------------------------------------------
# Sec. 4.2.9: contractions for the new local tensor
# ----------------------------------------------------------------------------

def _contract_axis(x: np.ndarray, axis: int, m: np.ndarray) -> np.ndarray:
    """Replace axis k of x by sum_k x[..k..] m[k, new], keeping its position."""
    y = np.tensordot(x, m, axes=([axis], [0]))
    return np.moveaxis(y, -1, axis)


def hat_matrix(tp: np.ndarray) -> np.ndarray:
    """The c-fixed tensors of every c0 as one matrix [(c0, n^..), (n^'.., rho)]
    (Sec. 3.2); loop-invariant in the contraction of Sec. 4.2.9."""
    d = tp.ndim // 2
    that = np.moveaxis(tp, 2 * d - 2, 0)       # [c0, n^.., n^'.., rho]
    rows = int(np.prod(that.shape[:d]))
    return np.ascontiguousarray(that).reshape(rows, -1)


def new_tensor_slab(tp: np.ndarray, us: list[np.ndarray], c0p: int, nprime: tuple,
                    that_mat: np.ndarray | None = None) -> np.ndarray:
    """Elements T^new_{n_{d-1}..n_1 n'_{d-1}..n'_1 c c'} for c' = c0p and one fixed
    n' = (n'_1, .., n'_{d-1}), for every c and n (Sec. 4.2.9).

    First step, Eqs. (TU1)-(TUNCD): prime-side chain on the c'-fixed tensor.
    Second step, Eq. (BottleneckPart): contraction with the c-fixed tensors over
    (n^', rho) -- done for all c0 at once.
    Last step, Eqs. (AfterBNNCD)-(AfterBN1): non-prime chain; Eq. (Elements_NewTensor).
    Returns an array [c, n_{d-1}, .., n_1].
    """
    d = tp.ndim // 2
    # c'-fixed tensor: T-check_{n.. n'.. rho} = T_{n.. n'.. rho c0p}
    tchk = tp[..., c0p]
    # first step: for j = 1..d-1 replace n-check'_j by n-hat'_j through
    # sum_{n-check'_j} U~^(j)_{(n^'_j n~'_j), n'_j} C~
    cchk = tchk
    for j in range(1, d):
        chi_j = int(round(math.sqrt(us[j - 1].shape[0])))
        u_col = us[j - 1][:, nprime[j - 1]].reshape(chi_j, chi_j)  # [n-check', n-hat']
        cchk = _contract_axis(cchk, _pos_np(d, j), u_col)
    # cchk axes: n~_{d-1}..n~_1, n^'_{d-1}..n^'_1, rho
    # second step (bottleneck): C^_{n~.. n^..} = sum_{n^', rho} T^_{n^.. n^'.. rho} C~_{n~.. n^'.. rho}
    # T-hat^{c=c0}_{n^.. n^'.. rho} = T_{n^.. n^'.. c0 rho}, all c0 at once, as the
    # matrix [(c0, n^..), (n^'.., rho)]; C~ as [(n~..), (n^'.., rho)]
    if that_mat is None:
        that_mat = hat_matrix(tp)
    chi_c = tp.shape[2 * d - 2]
    nchk = cchk.shape[: d - 1]
    chat = that_mat @ cchk.reshape(int(np.prod(nchk)), -1).T
    chat = chat.reshape((chi_c,) + tp.shape[: d - 1] + nchk)
    # chat axes: c0, n^_{d-1}..n^_1, n~_{d-1}..n~_1 -> paper order c0, n~.., n^..
    to_paper = [0] + list(range(d, 2 * d - 1)) + list(range(1, d))
    chat = np.transpose(chat, to_paper)
    # last step: for j = d-1 .. 1 contract (n^_j, n~_j) with U~^(j)_{(n^_j n~_j), n_j};
    # the new n_j joins the already formed n_{d-1}..n_{j+1} (Eqs. AfterBNNCD..AfterBN1)
    for j in range(d - 1, 0, -1):
        formed = d - 1 - j
        pos_chk = 1 + formed            # n~_j
        pos_hat = 1 + formed + j        # n^_j
        chi_j = int(round(math.sqrt(us[j - 1].shape[0])))
        u3 = us[j - 1].reshape(chi_j, chi_j, -1)   # [n~_j, n^_j, n_j]
        chat = np.tensordot(chat, u3, axes=([pos_chk, pos_hat], [0, 1]))
        chat = np.moveaxis(chat, -1, 1 + formed)
    return chat  # [c0, n_{d-1}, .., n_1]


def new_tensor(tp: np.ndarray, us: list[np.ndarray], progress=None) -> np.ndarray:
    """T^new in paper order, looping over c'_0 and over n'_1 (outermost) ..
    n'_{d-1} (innermost) as Sec. 4.2.9 prescribes (Eq. Elements_NewTensor)."""
    d = tp.ndim // 2
    chi_c = tp.shape[2 * d - 2]
    chi_new = [u.shape[1] for u in us]          # j = 1..d-1
    shape = [chi_new[j - 1] for j in range(d - 1, 0, -1)] * 2 + [chi_c, chi_c]
    out = np.zeros(shape)
    that_mat = hat_matrix(tp)
    for c0p in range(chi_c):
        for nprime in itertools.product(*[range(k) for k in chi_new]):
            slab = new_tensor_slab(tp, us, c0p, nprime, that_mat)   # [c0, n_{d-1}..n_1]
            idx = tuple(nprime[j - 1] for j in range(d - 1, 0, -1))
            # out[n_{d-1}..n_1, n'_{d-1}..n'_1, c, c'] = slab[c, n..]
            out[(Ellipsis,) + idx + (slice(None), c0p)] = np.moveaxis(slab, 0, -1)
            if progress is not None:
                progress()
    return out


# ----------------------------------------------------------------------------
# One coarse-graining and the run (Secs. 4.1.1, 4.2.1, 4.2.10-4.2.16)
# ----------------------------------------------------------------------------

@dataclass
class StepRecord:
    step: int
    axis: int
    chis: tuple               # bond dims per physical axis after the step
    trace: float              # Tr T^(p) of the new, not yet normalised tensor
    ln_z: float               # ln Z^(p) = K^(p) + ln Tr T^(p)   (Eq. eq_lnZ)
    ln_z_per_site: float      # ln Z^(p) / V^(p), V^(p) = 2^p
    gu_wen_x: float
    legs: list = field(default_factory=list)


def coarse_grain(t: np.ndarray, axis: int, chi: int):
    """One coarse-graining of a normalised tensor along physical `axis` with
    bond-dimension parameter chi.  Returns (T_new_unnormalised, legs, y)
    in the physical layout."""
    d = t.ndim // 2
    tp = to_paper_order(t, axis)
    nxt = next_axes(d, axis)
    legs = [choose_isometry(tp, j, chi, nxt[j - 1]) for j in range(1, d)]
    tnew_p = new_tensor(tp, [leg.u for leg in legs])
    y = y_matrix_paper(tnew_p)
    return from_paper_order(tnew_p, axis), legs, y


class HotrgRun:
    """A run of coarse-grainings with the bookkeeping of Secs. 4.1.1 and 4.2.1.

    ln Z^(0) = ln Tr T^(0) (p = 0, V = 1); before step q+1 the tensor is
    multiplied by f^(q) = 1 / Tr T^(q) and K^(q+1) = 2 (K^(q) + ln (f^(q))^-1).
    """

    def __init__(self, d: int, beta: float, h: float, tensor: np.ndarray | None = None):
        self.d = d
        self.beta = beta
        t = initial_tensor(d, beta, h) if tensor is None else np.array(tensor, dtype=np.float64)
        self.p = 0
        self.k = 0.0                                  # K^(0) = 0
        tr = trace_physical(t)
        self.trace0 = tr
        self.ln_z = self.k + math.log(tr)             # ln Z^(0)
        self.f = 1.0 / tr                             # f^(0)
        self.t = self.f * t                           # normalised before step 1
        self.records: list[StepRecord] = []

    @property
    def chis(self):
        return tuple(self.t.shape[2 * k] for k in range(self.d))

    def step(self, axis: int, chi: int) -> StepRecord:
        self.k = 2.0 * (self.k + math.log(1.0 / self.f))   # K^(p) (Eq. K_recurrence)
        tnew, legs, y = coarse_grain(self.t, axis, chi)
        self.p += 1
        tr = float(np.trace(y))                               # Tr T^(p) = trace Y
        if not (tr > 0.0 and math.isfinite(tr)):
            raise FloatingPointError(f"non-positive or non-finite trace {tr}")
        self.ln_z = self.k + math.log(tr)                     # Eq. eq_lnZ
        rec = StepRecord(self.p, axis, tuple(tnew.shape[2 * k] for k in range(self.d)),
                         tr, self.ln_z, self.ln_z / 2.0 ** self.p, gu_wen_ratio(y), legs)
        self.f = 1.0 / tr                                     # f^(p)
        self.t = self.f * tnew                                # normalisation (Sec. 4.2.16)
        self.records.append(rec)
        return rec

    def free_energy_per_site(self) -> float:
        """f = -(ln Z / V) / beta."""
        return -(self.ln_z / 2.0 ** self.p) / self.beta


def run(d: int, beta: float, h: float, chi: int, axes) -> list[StepRecord]:
    r = HotrgRun(d, beta, h)
    for a in axes:
        r.step(a, chi)
    return r.records


def cyclic_axes(d: int, nsteps: int, first: int = 0):
    """Axes cycling as in Sec. 3.1.2 (Next 1 becomes Current)."""
    return [(first + s) % d for s in range(nsteps)]
