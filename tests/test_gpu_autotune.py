"""The launch-shape autotuner of the chain stages (hotrg_set_autotune): it picks a grid
cap per stage shape from timed runs on the real operands, and the results are the same
bit for bit as without it."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2110_03607_gb300 as p

    p.load()
    return p


def _run(pkg, d, beta, h, chi, nsteps, tune):
    g = pkg.Hotrg(d, beta, h, precision=pkg.PREC_BF16X6, fp64_below=0.0)
    try:
        if tune:
            pkg.hotrg_set_autotune(g.ctx, True)
        lnz = []
        for s in range(nsteps):
            g.step((d - 1 + s) % d, chi)
            lnz.append(g.free_energy()[0])
        return lnz, pkg.hotrg_tensor(g.ctx), pkg.hotrg_autotune_entries(g.ctx)
    finally:
        g.close()


@pytest.mark.parametrize("d,beta,h,chi,nsteps", [(3, 0.2216544, 0.0, 8, 6), (3, 0.25, 0.05, 6, 5),
                                                 (2, 0.44, 0.0, 16, 8)])
def test_tuned_runs_equal_untuned_runs_bit_for_bit(pkg, d, beta, h, chi, nsteps):
    ref, t_ref, none = _run(pkg, d, beta, h, chi, nsteps, tune=False)
    got, t_got, choices = _run(pkg, d, beta, h, chi, nsteps, tune=True)
    assert none == []
    assert len(choices) > 0 and set(choices) <= {4, 8, 16, 32}
    assert got == ref
    np.testing.assert_array_equal(t_got, t_ref)


def test_autotune_arguments(pkg):
    g = pkg.Hotrg(2, 0.4, 0.0)
    try:
        assert pkg.load().hotrg_set_autotune(g.ctx, 2) == -1     # HOTRG_EINVAL
        assert pkg.hotrg_autotune_entries(g.ctx) == []
    finally:
        g.close()
