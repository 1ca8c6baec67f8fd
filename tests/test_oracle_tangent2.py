"""Pins of the second-derivative oracle (d^2/d beta^2 of a HOTRG run, specific heat)
against results fixed from outside it (no GPU): second differences along smooth paths,
central differences of the pinned first-derivative oracle, and exact enumeration of
small lattices (c = beta^2 Var(H) / N).
"""

import numpy as np
import pytest

from oracle import hotrg_oracle as o
from oracle import hotrg_tangent as tg
from oracle import hotrg_tangent2 as t2
from tests import exact_ising as ex


@pytest.mark.parametrize("d", [2, 3, 4])
@pytest.mark.parametrize("h", [0.0, 0.2])
def test_initial_tensor_second_derivative_matches_central_difference(d, h):
    beta, db = 0.37, 1e-5
    fd = (tg.initial_tensor_dbeta(d, beta + db, h) - tg.initial_tensor_dbeta(d, beta - db, h)) / (2 * db)
    np.testing.assert_allclose(t2.initial_tensor_d2beta(d, beta, h), fd, rtol=1e-7, atol=1e-8)


def _path(rng, shape):
    t = rng.standard_normal(shape)
    return t, rng.standard_normal(shape), rng.standard_normal(shape)


@pytest.mark.parametrize("prime", [False, True])
def test_environment_second_derivative_matches_second_difference(prime):
    # A(T) along T(e) = t + e dt + e^2/2 ddt: A''(0) by the second difference (A is a
    # polynomial of degree 4 in e, so the difference is exact up to e^2 terms)
    rng = np.random.default_rng(3)
    t, dt, ddt = _path(rng, (3,) * 6)
    e = 1e-3

    def a_at(x):
        return o.environment_matrix(t + x * dt + 0.5 * x * x * ddt, 1, prime)

    fd = (a_at(e) - 2 * a_at(0.0) + a_at(-e)) / (e * e)
    got = t2.environment_matrix_ddot(t, dt, ddt, 1, prime)
    np.testing.assert_allclose(got, fd, rtol=1e-5, atol=1e-5 * np.abs(fd).max())


def _sym(rng, n):
    x = rng.standard_normal((n, n))
    return x + x.T


def test_kept_isometry_derivatives_match_the_projector_along_a_path():
    # P(e) = U U^T of the leading 3 eigenvectors of A0 + e A1 + e^2/2 A2: P'(0) and P''(0)
    # by differences against the forms built from (U, dU, d2U); dU equals the first-order
    # oracle's
    rng = np.random.default_rng(5)
    n, k = 7, 3
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    a0 = q @ np.diag([9.0, 7.0, 5.5, 3.0, 2.0, 1.0, 0.5]) @ q.T
    a1, a2 = _sym(rng, n), _sym(rng, n)

    def proj(x):
        w, v = np.linalg.eigh(a0 + x * a1 + 0.5 * x * x * a2)
        u = v[:, np.argsort(w)[::-1][:k]]
        return u @ u.T

    lam, v = np.linalg.eigh(a0)
    order = np.argsort(lam)[::-1]
    lam, v = lam[order], v[:, order]
    u = v[:, :k]
    du, ddu, skipped = t2.kept_isometry_derivatives(lam, v, k, a1, a2)
    assert skipped == 0
    du1, _ = tg.kept_eigenvector_dot(lam, v, k, a1)
    np.testing.assert_allclose(du, du1, atol=1e-13)
    e = 1e-4
    p1_fd = (proj(e) - proj(-e)) / (2 * e)
    p2_fd = (proj(e) - 2 * proj(0.0) + proj(-e)) / (e * e)
    p1 = du @ u.T + u @ du.T
    p2 = ddu @ u.T + 2 * du @ du.T + u @ ddu.T
    np.testing.assert_allclose(p1, p1_fd, atol=1e-8)
    np.testing.assert_allclose(p2, p2_fd, atol=1e-5)
    # the parallel-transport gauge: no rotation inside the kept space
    np.testing.assert_allclose(u.T @ du, 0.0, atol=1e-13)


TRUNCATED = [
    (2, 0.35, 0.0, 6, 8),
    (2, 0.5, 0.05, 5, 8),
    (3, 0.2, 0.0, 3, 5),
    (3, 0.25, 0.1, 3, 4),
    (4, 0.15, 0.0, 2, 4),
]


def _dlnz(d, beta, h, chi, axes):
    r = tg.HotrgTangentRun(d, beta, h)
    for a in axes:
        rec = r.step(a, chi)
    return rec.dln_z_per_site


@pytest.mark.parametrize("d,beta,h,chi,nsteps", TRUNCATED)
def test_truncated_run_second_derivative_matches_central_difference(d, beta, h, chi, nsteps):
    axes = o.cyclic_axes(d, nsteps)
    r = t2.HotrgTangent2Run(d, beta, h)
    for a in axes:
        rec = r.step(a, chi)
    assert rec.degenerate_pairs == 0
    db = 1e-5
    fd = (_dlnz(d, beta + db, h, chi, axes) - _dlnz(d, beta - db, h, chi, axes)) / (2 * db)
    assert rec.d2ln_z_per_site == pytest.approx(fd, rel=2e-6)
    assert rec.dln_z_per_site == pytest.approx(_dlnz(d, beta, h, chi, axes), rel=1e-13)


@pytest.mark.parametrize("d,nsteps,chi,beta,h", [
    (2, 4, 16, 0.35, 0.0), (2, 4, 16, 0.3, 0.1), (2, 2, 4, 0.6, 0.02), (3, 3, 16, 0.25, 0.05),
])
def test_untruncated_specific_heat_equals_brute_force(d, nsteps, chi, beta, h):
    axes = o.cyclic_axes(d, nsteps, first=d - 1)
    r = t2.HotrgTangent2Run(d, beta, h)
    for i, a in enumerate(axes):
        rec = r.step(a, chi)
        exact = ex.brute_force_specific_heat(ex.lattice_after(d, axes[: i + 1]), beta, h)
        assert rec.specific_heat_per_site == pytest.approx(exact, rel=1e-10, abs=1e-13), i


def test_dropping_the_second_order_isometry_term_is_caught(monkeypatch):
    # planted mistake: d2U without the P' P' U term misses the central difference
    d, beta, h, chi, nsteps = TRUNCATED[0]
    axes = o.cyclic_axes(d, nsteps)
    real = t2.kept_isometry_derivatives

    def planted(lam, v, chi_new, da, dda):
        du, ddu, sk = real(lam, v, chi_new, da, dda)
        n = v.shape[0]
        g1 = v.T @ da @ v
        kept = np.arange(n) < chi_new
        p1 = np.zeros((n, n))
        for a in range(n):
            for c in range(n):
                if kept[a] != kept[c]:
                    p1[a, c] = (float(kept[a]) - float(kept[c])) / (lam[a] - lam[c]) * g1[a, c]
        return du, ddu - v @ (p1 @ p1)[:, :chi_new], sk

    monkeypatch.setattr(t2, "kept_isometry_derivatives", planted)
    r = t2.HotrgTangent2Run(d, beta, h)
    for a in axes:
        rec = r.step(a, chi)
    db = 1e-5
    fd = (_dlnz(d, beta + db, h, chi, axes) - _dlnz(d, beta - db, h, chi, axes)) / (2 * db)
    assert abs(rec.d2ln_z_per_site - fd) > 1e-5 * abs(fd)
