"""GPU second derivative d^2(ln Z/V)/d beta^2 (hotrg_set_tangent(ctx, 2), FP64 form) through
the C ABI against the second-derivative oracle, exact enumeration of untruncated lattices,
central differences of the GPU's own first derivative, and the double backward of the
torch.autograd interface."""

import numpy as np
import pytest

from oracle import hotrg_oracle as o
from oracle import hotrg_tangent2 as t2
from tests import exact_ising as ex

pytestmark = pytest.mark.gpu

ESTATE, EINVAL = -7, -1   # HOTRG_ESTATE, HOTRG_EINVAL (include/hotrg.h)


@pytest.fixture(scope="module")
def pkg():
    import torch

    import paper_2110_03607_gb300 as p

    assert torch.cuda.is_available()
    p.load()
    return p


def _gpu_run2(pkg, d, beta, h, chi, axes, order=2):
    g = pkg.Hotrg(d, beta, h, precision=pkg.PREC_FP64)
    out = []
    try:
        pkg.hotrg_set_tangent(g.ctx, order)
        for a in axes:
            g.step(a, chi)
            lnz, _ = g.free_energy()
            dlnz, _, deg = g.energy()
            d2 = g.specific_heat() if order == 2 else (None, None)
            out.append((lnz, dlnz, d2[0], d2[1], deg))
    finally:
        g.close()
    return out


CASES = [
    (2, 0.35, 0.0, 6, 8),
    (2, 0.5, 0.05, 5, 8),
    (3, 0.2, 0.0, 3, 5),
    (3, 0.25, 0.1, 3, 4),
    (4, 0.15, 0.0, 2, 4),
]


@pytest.mark.parametrize("d,beta,h,chi,nsteps", CASES)
def test_second_derivative_matches_oracle_every_step(pkg, d, beta, h, chi, nsteps):
    axes = o.cyclic_axes(d, nsteps)
    res = _gpu_run2(pkg, d, beta, h, chi, axes)
    first = _gpu_run2(pkg, d, beta, h, chi, axes, order=1)
    r = t2.HotrgTangent2Run(d, beta, h)
    for i, a in enumerate(axes):
        rec = r.step(a, chi)
        lnz, dlnz, d2, c, deg = res[i]
        assert deg == rec.degenerate_pairs == 0
        assert abs(lnz - rec.ln_z_per_site) <= 1e-12 * abs(rec.ln_z_per_site)
        assert abs(dlnz - rec.dln_z_per_site) <= 1e-10 * abs(rec.dln_z_per_site)
        assert abs(d2 - rec.d2ln_z_per_site) <= 1e-9 * abs(rec.d2ln_z_per_site), (i, d2, rec.d2ln_z_per_site)
        assert c == pytest.approx(beta * beta * d2, rel=1e-15)
        # carrying the second order leaves the first derivative as it was (to rounding:
        # its Grams are then dense, not in Z2 blocks)
        assert abs(dlnz - first[i][1]) <= 1e-12 * abs(dlnz)


@pytest.mark.parametrize("d,nsteps,chi,beta,h", [(2, 4, 16, 0.35, 0.0), (2, 4, 16, 0.3, 0.1),
                                                 (3, 3, 16, 0.25, 0.05)])
def test_untruncated_specific_heat_equals_brute_force(pkg, d, nsteps, chi, beta, h):
    axes = o.cyclic_axes(d, nsteps, first=d - 1)
    res = _gpu_run2(pkg, d, beta, h, chi, axes)
    for i in range(nsteps):
        exact = ex.brute_force_specific_heat(ex.lattice_after(d, axes[: i + 1]), beta, h)
        assert res[i][3] == pytest.approx(exact, rel=1e-10, abs=1e-13), i


@pytest.mark.parametrize("d,beta,h,chi,nsteps", [(3, 0.22, 0.0, 6, 6), (2, 0.44, 0.0, 12, 12)])
def test_second_derivative_matches_central_difference_of_the_gpu_first_derivative(pkg, d, beta, h, chi, nsteps):
    # beyond the oracle's sizes: the GPU's own FP64 first derivative at beta +- 1e-5
    axes = o.cyclic_axes(d, nsteps)
    d2 = _gpu_run2(pkg, d, beta, h, chi, axes)[-1][2]
    db = 1e-5
    up = _gpu_run2(pkg, d, beta + db, h, chi, axes, order=1)[-1][1]
    dn = _gpu_run2(pkg, d, beta - db, h, chi, axes, order=1)[-1][1]
    fd = (up - dn) / (2 * db)
    assert abs(d2 - fd) <= 5e-6 * abs(fd), (d2, fd)


def test_autograd_double_backward_gives_the_second_derivative(pkg):
    import torch

    from paper_2110_03607_gb300 import autograd as ag

    d, beta, h, chi = 3, 0.22, 0.0, 3
    axes = o.cyclic_axes(d, 5, first=2)
    bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    lnz = ag.ln_z_per_site(bt, d, h, chi, axes, order=2)
    r = t2.HotrgTangent2Run(d, beta, h)
    recs = [r.step(a, chi) for a in axes]
    (g,) = torch.autograd.grad(lnz[-1], bt, create_graph=True)
    (g2,) = torch.autograd.grad(g, bt)
    assert abs(float(g.detach()) - recs[-1].dln_z_per_site) <= 1e-10 * abs(recs[-1].dln_z_per_site)
    assert abs(float(g2) - recs[-1].d2ln_z_per_site) <= 1e-9 * abs(recs[-1].d2ln_z_per_site)
    c = ag.specific_heat_per_site(beta, d, h, chi, axes)
    assert c == pytest.approx(recs[-1].specific_heat_per_site, rel=1e-9)
    # first order only: the gradient is not differentiable again
    lnz1 = ag.ln_z_per_site(torch.tensor(beta, dtype=torch.float64, requires_grad=True), d, h, chi, axes,
                            pkg.PREC_BF16X6)
    with pytest.raises(ValueError):
        ag.ln_z_per_site(bt, d, h, chi, axes, pkg.PREC_BF16X6, order=2)
    assert lnz1.shape == lnz.shape


def test_second_order_refusals(pkg):
    g = pkg.Hotrg(2, 0.4, 0.0, precision=pkg.PREC_BF16X6)
    try:
        with pytest.raises(pkg.HotrgError) as e:      # split precision
            pkg.hotrg_set_tangent(g.ctx, 2)
        assert e.value.status == EINVAL
        with pytest.raises(pkg.HotrgError) as e:      # not carried
            g.specific_heat()
        assert e.value.status == ESTATE
    finally:
        g.close()
    g = pkg.Hotrg(2, 0.4, 0.0, precision=pkg.PREC_FP64)
    try:
        pkg.hotrg_set_tangent(g.ctx, 2)
        with pytest.raises(pkg.HotrgError) as e:      # the FP64 form is kept
            pkg.hotrg_set_precision(g.ctx, pkg.PREC_BF16X6)
        assert e.value.status == EINVAL
        g.step(0, 4)
        assert np.isfinite(g.specific_heat()[1])
    finally:
        g.close()
