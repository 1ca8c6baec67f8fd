"""Pins of the FP64 oracle against results fixed from outside it (no GPU).

Each test checks the oracle against something other than itself: exact
enumeration, transfer matrices, Onsager's solution, the high-temperature
series, the paper's own definitions written out a second way (explicit M),
a library eigen-solver, and invariants (isometry, Z2, K recurrence).  The last
tests plant plausible mistakes in the oracle (a sign, an index, a transposed
operand, the wrong end of the spectrum) and check that a pin catches each.
"""

import math

import numpy as np
import pytest

from oracle import hotrg_oracle as o
from tests import exact_ising as ex

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


# ---------------------------------------------------------------------------
# Initial tensor (Sec. 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("beta", [0.0, 0.1, 0.4406868, 1.3])
def test_factor_matrix_reproduces_boltzmann_weight(beta):
    x = o.ising_factor_matrix(beta)
    s = np.array([1.0, -1.0])
    w = np.exp(beta * np.outer(s, s))
    np.testing.assert_allclose(x @ x.T, w, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_initial_tensor_closed_form(d):
    beta, h = 0.37, 0.2
    t = o.initial_tensor(d, beta, h)
    ch, sh = math.cosh(beta), math.sinh(beta)
    for idx in [(0,) * (2 * d), (1, 1) + (0,) * (2 * d - 2), (1,) * (2 * d), (1,) + (0,) * (2 * d - 1)]:
        k = sum(idx)
        # sum_s V_s prod_legs X_{s j}: X_{s0} = sqrt(cosh), X_{s1} = +-sqrt(sinh)
        want = sum(math.exp(beta * h * sg) * (sg ** k) for sg in (1.0, -1.0)) \
            * ch ** ((2 * d - k) / 2) * sh ** (k / 2)
        assert t[idx] == pytest.approx(want, rel=1e-14)


# ---------------------------------------------------------------------------
# Exactness without truncation (Sec. 2: chi_s^2 <= chi keeps U square)
# ---------------------------------------------------------------------------

EXACT_CASES = [
    (2, 2, 4), (2, 4, 16), (3, 3, 16),
    (4, 2, 16),     # 4D: axes w, x -> the periodic 2 x 1 x 1 x 2 lattice, bonds (4, 16, 16, 4)
]


@pytest.mark.parametrize("d,nsteps,chi", EXACT_CASES)
@pytest.mark.parametrize("beta", [0.1, 0.22, 0.44])
@pytest.mark.parametrize("h", [0.0, 0.01, 0.3])
def test_untruncated_run_equals_brute_force(d, nsteps, chi, beta, h):
    axes = o.cyclic_axes(d, nsteps, first=d - 1)
    r = o.HotrgRun(d, beta, h)
    assert r.ln_z == pytest.approx(ex.brute_force_ln_z((1,) * d, beta, h), rel=1e-13)
    for i, a in enumerate(axes):
        rec = r.step(a, chi)
        exact = ex.brute_force_ln_z(ex.lattice_after(d, axes[: i + 1]), beta, h)
        assert rec.ln_z == pytest.approx(exact, rel=1e-12), (i, rec.chis)


@pytest.mark.parametrize("beta,h", [(0.3, 0.0), (0.44, 0.3)])
def test_transfer_matrices_agree_with_enumeration_and_oracle(beta, h):
    tm2 = ex.transfer_matrix_ln_z_2d(4, 4, beta, h)
    assert tm2 == pytest.approx(ex.brute_force_ln_z((4, 4), beta, h), rel=1e-13)
    tm3 = ex.transfer_matrix_ln_z_3d(2, 2, 2, beta, h)
    assert tm3 == pytest.approx(ex.brute_force_ln_z((2, 2, 2), beta, h), rel=1e-13)
    r = o.HotrgRun(2, beta, h)
    for a in o.cyclic_axes(2, 4):
        rec = r.step(a, 16)
    assert rec.ln_z == pytest.approx(tm2, rel=1e-12)
    r = o.HotrgRun(3, beta, h)
    for a in o.cyclic_axes(3, 3):
        rec = r.step(a, 16)
    assert rec.ln_z == pytest.approx(tm3, rel=1e-12)


@pytest.mark.parametrize("d,chi,nsteps", [(2, 3, 8), (3, 3, 6), (4, 2, 5)])
def test_beta_zero_is_ln2_per_site(d, chi, nsteps):
    # beta = 0: T0 has the single entry 2 at all-zero legs, Z = 2^V
    r = o.HotrgRun(d, 0.0, 0.0)
    for a in o.cyclic_axes(d, nsteps):
        rec = r.step(a, chi)
        assert rec.ln_z_per_site == pytest.approx(math.log(2.0), rel=1e-14)


# ---------------------------------------------------------------------------
# Truncated runs against closed forms
# ---------------------------------------------------------------------------

def test_high_temperature_series_2d():
    # ln Z/N = ln 2 + 2 ln cosh b + t^4 + 2 t^6 + O(t^8) on the square lattice
    beta = 0.05
    t = math.tanh(beta)
    r = o.HotrgRun(2, beta, 0.0)
    for a in o.cyclic_axes(2, 12):
        rec = r.step(a, 8)
    series = ex.high_t_series(2, beta) + 2 * t ** 6
    assert abs(rec.ln_z_per_site - series) <= 10 * t ** 8


def test_high_temperature_series_3d():
    # 3t^4 + 22t^6 (polygons of 4 and 6 bonds per site of the cubic lattice);
    # chi = 6 HOTRG truncation leaves an error ~1e-6 here, so the gate is loose
    beta = 0.05
    t = math.tanh(beta)
    r = o.HotrgRun(3, beta, 0.0)
    for a in o.cyclic_axes(3, 9):
        rec = r.step(a, 6)
    series = ex.high_t_series(3, beta) + 22 * t ** 6
    assert abs(rec.ln_z_per_site - series) <= 3e-6
    # dropping the plaquette term is caught
    assert abs(rec.ln_z_per_site - (series - 3 * t ** 4)) > 1e-5


def test_onsager_forms_agree():
    for beta in (0.3, 0.5):
        assert ex.onsager_ln_z_per_site(beta) == pytest.approx(ex.onsager_double_integral(beta), rel=1e-12)


@pytest.mark.parametrize("beta,gate,ordered", [(0.3, 1e-6, False), (0.4406868, 1e-4, False), (0.5, 1e-5, True)])
def test_onsager_chi8_20_steps(beta, gate, ordered):
    r = o.HotrgRun(2, beta, 0.0)
    for a in o.cyclic_axes(2, 20):
        rec = r.step(a, 8)
    exact = ex.onsager_ln_z_per_site(beta)
    if ordered:
        # two degenerate ground states of a finite periodic lattice add ln 2 / N
        exact += math.log(2.0) / 2 ** 20
    assert abs(rec.ln_z_per_site - exact) / exact <= gate
    # Gu-Wen ratio (Sec. 4.1.2): 1 in the disordered phase, m = 2 in the Z2-broken phase
    if beta != 0.4406868:
        assert rec.gu_wen_x == pytest.approx(2.0 if ordered else 1.0, abs=1e-3)


def test_onsager_error_shrinks_with_chi_at_criticality():
    beta = 0.4406868
    exact = ex.onsager_ln_z_per_site(beta)
    errs = []
    for chi in (6, 10):
        r = o.HotrgRun(2, beta, 0.0)
        for a in o.cyclic_axes(2, 16):
            rec = r.step(a, chi)
        errs.append(abs(rec.ln_z_per_site - exact))
    assert errs[1] < errs[0]


# ---------------------------------------------------------------------------
# The paper's definitions written out a second way
# ---------------------------------------------------------------------------

def _explicit_m(tp):
    """M of Sec. 2 from its definition, axes (n^_k, n~_k) pairs then c, c'."""
    d = tp.ndim // 2
    letters = "abcdefghijklmnop"
    hat = letters[: 2 * d - 2]
    chk = letters[2 * d - 2: 4 * d - 4]
    sub_hat = hat + "xr"
    sub_chk = chk + "ry"
    out = "".join(h + c for h, c in zip(hat, chk)) + "xy"
    return np.einsum(f"{sub_hat},{sub_chk}->{out}", tp, tp)


@pytest.mark.parametrize("d,chi,axis", [(2, 3, 0), (3, 5, 0), (3, 3, 1), (4, 3, 0), (4, 5, 2)])
def test_environment_truncation_and_new_tensor_match_definitions(d, chi, axis):
    r = o.HotrgRun(d, 0.3, 0.1)
    r.step((axis + d - 1) % d, 16)          # grow some bonds first
    _check_definitions(o.to_paper_order(r.t, axis), chi)


@pytest.mark.parametrize("chis,chi,seed", [([3, 3], 4, 0), ([3, 2], 3, 1), ([2, 3, 2], 3, 2), ([3, 2, 2], 5, 3)])
def test_definitions_hold_on_a_tensor_without_reflection_symmetry(chis, chi, seed):
    # a Gaussian tensor has no lattice symmetry: S^ != S~ and A != A', so a mistake that
    # swaps the copies (c for c', hat for check) cannot cancel out
    import seeded_inputs as si
    _check_definitions(o.to_paper_order(si.gaussian_tensor(chis, seed), 0), chi)


def _check_definitions(tp, chi):
    """A, A', the truncation identity and T_new of the oracle against explicit M (Sec. 2)."""
    d = tp.ndim // 2
    m = _explicit_m(tp)
    legs = [o.choose_isometry(tp, j, chi, None) for j in range(1, d)]
    us = [leg.u for leg in legs]
    for j in range(1, d):
        for prime in (False, True):
            pos = 2 * (o._pos_np(d, j) if prime else o._pos_n(d, j))
            mt = np.moveaxis(m, [pos + 1, pos], [0, 1])   # [check, hat, rest]
            cj = mt.shape[0]
            mt = mt.reshape(cj * cj, -1)
            a_def = mt @ mt.T
            a_or = o.environment_matrix(tp, j, prime)
            np.testing.assert_allclose(a_or, a_def, rtol=0, atol=1e-13 * np.abs(a_def).max())
            leg = legs[j - 1]
            if prime == leg.chose_prime:
                # HOSVD truncation identity: ||M~ - U U^T M~||^2 = sum of discarded eigenvalues
                resid = mt - leg.u @ (leg.u.T @ mt)
                eps = leg.eps_prime if prime else leg.eps
                assert (resid ** 2).sum() == pytest.approx(eps, rel=1e-8, abs=1e-14 * np.abs(a_def).max())
    # Eq. (CoarseGrainingProcedure_d): U~ ... M ... U~ against the chain of Sec. 4.2.9
    sub = ""
    ops = [m]
    letters = "abcdefghijklmnop"
    pair_letters = letters[: 4 * d - 4]
    new_unp = "ABCDEFG"[: d - 1]
    new_pri = "HIJKLMN"[: d - 1]
    m_sub = pair_letters + "xy"
    u_subs = []
    for k in range(2 * d - 2):
        hat_l, chk_l = pair_letters[2 * k], pair_letters[2 * k + 1]
        # pair k: k < d-1 -> n_{d-1-k}, else n'_{2d-2-1-k}
        if k < d - 1:
            j = d - 1 - k
            new_l = new_unp[k]
        else:
            j = 2 * d - 2 - k
            new_l = new_pri[k - (d - 1)]
        cj = int(round(math.sqrt(us[j - 1].shape[0])))
        ops.append(us[j - 1].reshape(cj, cj, -1))   # [check, hat, new]
        u_subs.append(chk_l + hat_l + new_l)
    expr = m_sub + "," + ",".join(u_subs) + "->" + new_unp + new_pri + "xy"
    t_def = np.einsum(expr, *ops, optimize=True)
    t_chain = o.new_tensor(tp, us)
    np.testing.assert_allclose(t_chain, t_def, rtol=0, atol=1e-12 * np.abs(t_def).max())


def test_k_recurrence_matches_direct_sum():
    # K^(p) = sum_{l<p} 2^(p-l) ln (f^(l))^-1 (Eq. eq_lnZ) against the recurrence (Eq. K_recurrence)
    r = o.HotrgRun(2, 0.4, 0.05)
    traces = [r.trace0]
    for a in o.cyclic_axes(2, 8):
        rec = r.step(a, 6)
        k_direct = sum(2.0 ** (r.p - l) * math.log(traces[l]) for l in range(r.p))
        assert rec.ln_z - math.log(rec.trace) == pytest.approx(k_direct, rel=1e-14)
        traces.append(rec.trace)


# ---------------------------------------------------------------------------
# Invariants: isometry, Z2 zeros, eigen-solver
# ---------------------------------------------------------------------------

def test_isometries_are_isometric():
    r = o.HotrgRun(3, 0.2216544, 0.0)
    for a in o.cyclic_axes(3, 5):
        rec = r.step(a, 6)
        for leg in rec.legs:
            k = leg.u.shape[1]
            np.testing.assert_allclose(leg.u.T @ leg.u, np.eye(k), rtol=0, atol=1e-12)


@pytest.mark.parametrize("d,chi,beta", [(2, 8, 0.5), (3, 5, 0.2216544)])
def test_z2_odd_elements_vanish_at_zero_field(d, chi, beta):
    r = o.HotrgRun(d, beta, 0.0)
    parity = [np.array([0, 1])] * d          # index 0 even, index 1 odd (columns of X)
    for a in o.cyclic_axes(d, 3 * d):
        rec = r.step(a, chi)
        new_par = list(parity)
        for leg in rec.legs:
            pj = parity[leg.axis]
            cj = len(pj)
            row_par = (pj[None, :] + pj[:, None]) % 2     # [check, hat] -> row hat + check*cj
            row_par = row_par.reshape(-1)
            cols = []
            for k in range(leg.u.shape[1]):
                support = np.abs(leg.u[:, k]) > 1e-14
                ps = set(row_par[support].tolist())
                assert len(ps) == 1, "isometry column of indefinite parity"
                cols.append(ps.pop())
            new_par[leg.axis] = np.array(cols)
        parity = new_par
        t = r.t
        tot = np.zeros(t.shape, dtype=int)
        for k in range(d):
            for side in (0, 1):
                shape = [1] * (2 * d)
                shape[2 * k + side] = t.shape[2 * k + side]
                tot = tot + parity[k].reshape(shape)
        odd = (tot % 2) == 1
        assert np.abs(t[odd]).max(initial=0.0) <= 1e-12 * np.abs(t).max()


def test_jacobi_against_lapack_on_random_spd():
    rng = np.random.default_rng(7)
    for n in (1, 2, 5, 16, 37):
        g = rng.standard_normal((n, n + 3))
        a = g @ g.T
        lam, v, _ = o.sorted_eigenpairs(a)
        ref = np.linalg.eigvalsh(a)[::-1]
        np.testing.assert_allclose(lam, ref, rtol=0, atol=1e-12 * ref[0])
        np.testing.assert_allclose(v.T @ v, np.eye(n), rtol=0, atol=1e-12)
        np.testing.assert_allclose(v @ np.diag(lam) @ v.T, a, rtol=0, atol=1e-12 * ref[0])
        assert np.all(np.diff(lam) <= 0)


def test_jacobi_on_rank_deficient_environment_matrix():
    r = o.HotrgRun(2, 0.5, 0.0)
    for a in o.cyclic_axes(2, 10):
        r.step(a, 8)
    tp = o.to_paper_order(r.t, 0)
    a = o.environment_matrix(tp, 1, False)
    lam, v, _ = o.sorted_eigenpairs(a)
    ref = np.linalg.eigvalsh(a)[::-1]
    np.testing.assert_allclose(lam, np.maximum(ref, 0), rtol=0, atol=1e-12 * ref[0])
    np.testing.assert_allclose(v.T @ v, np.eye(a.shape[0]), rtol=0, atol=1e-12)


def test_sign_gauge_and_tie_order():
    # a matrix with an exactly degenerate pair: the tie is ordered by pivot index
    q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((4, 4)))
    a = q @ np.diag([3.0, 1.0, 1.0, 0.5]) @ q.T
    lam, v, _ = o.sorted_eigenpairs(a)
    np.testing.assert_allclose(lam, [3.0, 1.0, 1.0, 0.5], atol=1e-13)
    for k in range(4):
        assert v[o.pivot_index(v[:, k]), k] > 0
    assert o.pivot_index(v[:, 1]) <= o.pivot_index(v[:, 2])


def test_choice_rule_picks_smaller_discarded_sum():
    # Sec. 2 criterion: U if epsilon < epsilon', else U'.  A random tensor has no
    # reflection symmetry, so A and A' differ; the eigenvalues come from LAPACK here.
    import seeded_inputs as si
    for seed in range(6):
        t = si.gaussian_tensor([3, 3], seed)
        tp = o.to_paper_order(t, 0)
        leg = o.choose_isometry(tp, 1, 4, 1)
        lam = np.maximum(np.linalg.eigvalsh(o.environment_matrix(tp, 1, False))[::-1], 0)
        lamp = np.maximum(np.linalg.eigvalsh(o.environment_matrix(tp, 1, True))[::-1], 0)
        eps, epsp = lam[4:].sum(), lamp[4:].sum()
        assert abs(eps - epsp) > 1e-6 * lam[0]
        assert leg.chose_prime == (eps >= epsp)
        # the kept columns span the top eigenspace of the chosen side
        a = o.environment_matrix(tp, 1, leg.chose_prime)
        w, v = np.linalg.eigh(a)
        top = v[:, ::-1][:, :4]
        np.testing.assert_allclose(np.abs(np.linalg.svd(top.T @ leg.u)[1]), 1.0, atol=1e-10)


# ---------------------------------------------------------------------------
# Planted mistakes: each plausible error in the oracle fails one of the pins above
# ---------------------------------------------------------------------------

def test_planted_sign_error_in_the_factor_matrix_fails_the_enumeration_pins(monkeypatch):
    real = o.ising_factor_matrix

    def planted(beta):
        x = real(beta).copy()
        x[1, 1] = -x[1, 1]          # sigma_1 carries +sqrt(sinh) instead of -sqrt(sinh)
        return x

    monkeypatch.setattr(o, "ising_factor_matrix", planted)
    r = o.HotrgRun(2, 0.3, 0.1)
    rec = r.step(1, 4)
    exact = ex.brute_force_ln_z(ex.lattice_after(2, [1]), 0.3, 0.1)
    assert abs(rec.ln_z - exact) > 1e-3 * abs(exact)


def test_planted_index_mistake_in_the_environment_fails_the_definition_pin(monkeypatch):
    # S~ summed over c' instead of c (the Gram of the hat copy taken twice)
    import seeded_inputs as si
    real = o._gram

    def planted(tp, keep):
        d = tp.ndim // 2
        return real(tp, [2 * d - 1 if k == 2 * d - 2 else k for k in keep])

    monkeypatch.setattr(o, "_gram", planted)
    tp = o.to_paper_order(si.gaussian_tensor([3, 3], 0), 0)
    with pytest.raises(AssertionError):
        _check_definitions(tp, 4)


def test_planted_transposed_isometry_fails_the_definition_pin(monkeypatch):
    # the contraction reading U~ with (hat, check) swapped
    import seeded_inputs as si
    real = o.new_tensor

    def planted(tp, us, progress=None):
        swapped = []
        for u in us:
            c = int(round(math.sqrt(u.shape[0])))
            swapped.append(u.reshape(c, c, -1).transpose(1, 0, 2).reshape(c * c, -1))
        return real(tp, swapped, progress)

    monkeypatch.setattr(o, "new_tensor", planted)
    tp = o.to_paper_order(si.gaussian_tensor([3, 3], 0), 0)
    with pytest.raises(AssertionError):
        _check_definitions(tp, 4)


def test_planted_wrong_end_of_the_spectrum_fails_onsager(monkeypatch):
    # isometries built from the smallest eigenvalues instead of the largest
    real = o.sorted_eigenpairs

    def planted(a):
        lam, v, sw = real(a)
        return lam[::-1].copy(), v[:, ::-1].copy(), sw

    monkeypatch.setattr(o, "sorted_eigenpairs", planted)
    beta = 0.3
    exact = ex.onsager_ln_z_per_site(beta)
    try:
        r = o.HotrgRun(2, beta, 0.0)
        for a in o.cyclic_axes(2, 20):
            rec = r.step(a, 8)
        err = abs(rec.ln_z_per_site - exact) / exact
    except FloatingPointError:      # the kept space can lose the whole trace
        err = math.inf
    assert err > 1e-6
