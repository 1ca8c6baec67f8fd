"""Pins of the FP64 tangent oracle (d/d beta of a HOTRG run) against results fixed
from outside it (no GPU): finite differences of the pinned forward oracle, exact
enumeration of small lattices, Onsager's internal energy, and the forward
oracle's own new-tensor loop.
"""


import numpy as np
import pytest

from oracle import hotrg_oracle as o
from oracle import hotrg_tangent as tg
from tests import exact_ising as ex

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


def _normalised_tensor(d, beta, h, chi, nsteps):
    r = o.HotrgRun(d, beta, h)
    for a in o.cyclic_axes(d, nsteps):
        r.step(a, chi)
    return r.t, nsteps % d


@pytest.mark.parametrize("d", [2, 3, 4])
@pytest.mark.parametrize("h", [0.0, 0.2])
def test_initial_tensor_derivative_matches_central_difference(d, h):
    beta, db = 0.37, 1e-5
    fd = (o.initial_tensor(d, beta + db, h) - o.initial_tensor(d, beta - db, h)) / (2 * db)
    np.testing.assert_allclose(tg.initial_tensor_dbeta(d, beta, h), fd, rtol=1e-8, atol=1e-9)


def test_initial_tensor_derivative_needs_positive_beta():
    with pytest.raises(ValueError):
        tg.initial_tensor_dbeta(2, 0.0, 0.0)


@pytest.mark.parametrize("d,chi,nsteps", [(2, 4, 3), (3, 3, 2), (4, 2, 2)])
def test_one_einsum_form_equals_the_sliced_new_tensor(d, chi, nsteps):
    # contract_new with equal operands must reproduce the pinned slab loop of Sec. 4.2.9
    t, axis = _normalised_tensor(d, 0.4, 0.05, chi, nsteps)
    tp = o.to_paper_order(t, axis)
    nxt = o.next_axes(d, axis)
    us = [o.choose_isometry(tp, j, chi, nxt[j - 1]).u for j in range(1, d)]
    want = o.new_tensor(tp, us)
    got = tg.contract_new(tp, tp, us, us)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.abs(want).max())


@pytest.mark.parametrize("d,chi,nsteps", [(2, 4, 3), (3, 3, 2)])
def test_product_rule_of_the_new_tensor_matches_central_difference(d, chi, nsteps):
    # the contraction is multilinear: d along (dT, dU) by central differences
    rng = np.random.default_rng(7)
    t, axis = _normalised_tensor(d, 0.4, 0.05, chi, nsteps)
    tp = o.to_paper_order(t, axis)
    nxt = o.next_axes(d, axis)
    us = [o.choose_isometry(tp, j, chi, nxt[j - 1]).u for j in range(1, d)]
    dtp = rng.standard_normal(tp.shape)
    dus = [rng.standard_normal(u.shape) for u in us]
    e = 1e-4

    def at(s):
        return o.new_tensor(tp + s * dtp, [u + s * du for u, du in zip(us, dus)])

    fd = (at(e) - at(-e)) / (2 * e)
    got = tg.new_tensor_dot(tp, dtp, us, dus)
    np.testing.assert_allclose(got, fd, rtol=0, atol=1e-6 * np.abs(fd).max())


@pytest.mark.parametrize("prime", [False, True])
def test_environment_derivative_matches_central_difference(prime):
    d, chi = 3, 3
    rng = np.random.default_rng(3)
    t, axis = _normalised_tensor(d, 0.3, 0.0, chi, 2)
    tp = o.to_paper_order(t, axis)
    dtp = rng.standard_normal(tp.shape) * np.abs(tp).max()
    e = 1e-5
    for j in (1, 2):
        fd = (o.environment_matrix(tp + e * dtp, j, prime) - o.environment_matrix(tp - e * dtp, j, prime)) / (2 * e)
        got = tg.environment_matrix_dot(tp, dtp, j, prime)
        np.testing.assert_allclose(got, fd, rtol=0, atol=1e-7 * np.abs(fd).max())


def test_kept_subspace_derivative_matches_central_difference():
    # the kept projector P = U U^T is gauge free: dP = dU U^T + U dU^T by differences
    rng = np.random.default_rng(11)
    n, keep = 12, 5
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    a = q @ np.diag(np.linspace(10.0, 0.5, n)) @ q.T
    da = rng.standard_normal((n, n))
    da = da + da.T
    lam, v, _ = o.sorted_eigenpairs(a)
    du, skipped = tg.kept_eigenvector_dot(lam, v, keep, da)
    assert skipped == 0
    u = v[:, :keep]
    e = 1e-6

    def proj(s):
        _, vs, _ = o.sorted_eigenpairs(a + s * da)
        return vs[:, :keep] @ vs[:, :keep].T

    fd = (proj(e) - proj(-e)) / (2 * e)
    np.testing.assert_allclose(du @ u.T + u @ du.T, fd, rtol=0, atol=1e-7)
    # dU has no component inside the kept subspace
    np.testing.assert_allclose(u.T @ du, 0.0, atol=1e-12)


def test_degenerate_pair_across_the_cut_is_left_out_and_counted():
    lam = np.array([3.0, 2.0, 2.0, 1.0])
    v = np.eye(4)
    da = np.ones((4, 4))
    du, skipped = tg.kept_eigenvector_dot(lam, v, 2, da)
    assert skipped == 1
    assert np.all(np.isfinite(du))


def _ln_z_per_site(d, beta, h, chi, axes):
    r = o.HotrgRun(d, beta, h)
    for a in axes:
        r.step(a, chi)
    return r.ln_z / 2 ** r.p


TRUNCATED_CASES = [
    (2, 0.35, 0.0, 8, 10),
    (2, 0.5, 0.05, 6, 10),
    (3, 0.2, 0.0, 4, 6),
    (3, 0.25, 0.1, 4, 5),
    (4, 0.15, 0.0, 3, 4),
]


@pytest.mark.parametrize("d,beta,h,chi,nsteps", TRUNCATED_CASES)
def test_truncated_run_derivative_matches_central_difference(d, beta, h, chi, nsteps):
    axes = o.cyclic_axes(d, nsteps)
    r = tg.HotrgTangentRun(d, beta, h)
    for a in axes:
        rec = r.step(a, chi)
    assert rec.degenerate_pairs == 0
    db = 1e-5
    fd = (_ln_z_per_site(d, beta + db, h, chi, axes) - _ln_z_per_site(d, beta - db, h, chi, axes)) / (2 * db)
    assert rec.dln_z_per_site == pytest.approx(fd, rel=1e-7)
    assert rec.ln_z_per_site == pytest.approx(_ln_z_per_site(d, beta, h, chi, axes), rel=1e-14)


@pytest.mark.parametrize("d,beta,h,chi,nsteps", TRUNCATED_CASES[:4])
def test_dropping_the_isometry_derivative_is_caught(d, beta, h, chi, nsteps):
    # planted mistake: without dU the derivative misses the finite difference
    axes = o.cyclic_axes(d, nsteps)
    r = tg.HotrgTangentRun(d, beta, h, drop_du=True)
    for a in axes:
        rec = r.step(a, chi)
    db = 1e-5
    fd = (_ln_z_per_site(d, beta + db, h, chi, axes) - _ln_z_per_site(d, beta - db, h, chi, axes)) / (2 * db)
    assert abs(rec.dln_z_per_site - fd) > 1e-5 * abs(fd)


@pytest.mark.parametrize("d,nsteps,shape_chi,beta,h", [
    (2, 4, 16, 0.3, 0.1), (2, 4, 16, 0.44, 0.0), (2, 4, 16, 0.8, 0.02),
    (2, 2, 4, 0.3, 0.1), (3, 3, 16, 0.25, 0.05),
])
def test_untruncated_energy_equals_brute_force(d, nsteps, shape_chi, beta, h):
    axes = o.cyclic_axes(d, nsteps, first=d - 1)
    r = tg.HotrgTangentRun(d, beta, h)
    assert -r.dln_z == pytest.approx(ex.brute_force_energy((1,) * d, beta, h), rel=1e-13)
    for i, a in enumerate(axes):
        rec = r.step(a, shape_chi)
        exact = ex.brute_force_energy(ex.lattice_after(d, axes[: i + 1]), beta, h)
        assert rec.energy_per_site == pytest.approx(exact, rel=1e-11, abs=1e-13), i


def test_onsager_energy_closed_form_is_the_derivative_of_ln_z():
    for beta in (0.3, 0.5):
        db = 1e-5
        fd = -(ex.onsager_ln_z_per_site(beta + db) - ex.onsager_ln_z_per_site(beta - db)) / (2 * db)
        assert ex.onsager_energy_per_site(beta) == pytest.approx(fd, rel=1e-8)


@pytest.mark.parametrize("beta,gate", [(0.3, 1e-5), (0.5, 5e-5)])
def test_energy_chi8_20_steps_against_onsager(beta, gate):
    r = tg.HotrgTangentRun(2, beta, 0.0)
    for a in o.cyclic_axes(2, 20):
        rec = r.step(a, 8)
    exact = ex.onsager_energy_per_site(beta)
    assert abs(rec.energy_per_site - exact) / abs(exact) <= gate
    # a sign error or the missing 1/V would be far outside the gate
    assert abs(-rec.energy_per_site - exact) / abs(exact) > 1.0


@pytest.mark.parametrize("d,nsteps,chi,beta,h", [(2, 4, 16, 0.35, 0.0), (3, 3, 16, 0.25, 0.05)])
def test_specific_heat_from_energies_equals_brute_force(d, nsteps, chi, beta, h):
    # c = -beta^2 du/dbeta from central differences of the tangent run's energy (the way
    # the beta scan reports it), on lattices the run builds without truncation
    axes = o.cyclic_axes(d, nsteps, first=d - 1)
    db = 1e-4

    def energy(b):
        r = tg.HotrgTangentRun(d, b, h)
        for a in axes:
            rec = r.step(a, chi)
        return rec.energy_per_site

    c = -beta ** 2 * (energy(beta + db) - energy(beta - db)) / (2 * db)
    exact = ex.brute_force_specific_heat(ex.lattice_after(d, axes), beta, h)
    assert c == pytest.approx(exact, rel=1e-6)
