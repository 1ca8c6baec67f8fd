"""Captured steps (hotrg_graph_capture / hotrg_graph_launch): a replayed cycle of steps
gives the uncaptured run's results bit for bit, and the captures that cannot be replayed
are refused."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ESTATE, EINVAL = -7, -1   # HOTRG_ESTATE, HOTRG_EINVAL (include/hotrg.h)


@pytest.fixture(scope="module")
def pkg():
    import paper_2110_03607_gb300 as p

    p.load()
    return p


def _axes(d, n, first):
    return [(first + s) % d for s in range(n)]


def _state(pkg, g):
    lnz, _ = g.free_energy()
    tr, x, p = pkg.hotrg_observables(g.ctx)
    return lnz, tr, x, p, pkg.hotrg_tensor(g.ctx)


# d, beta, h, chi, precision, forget parities (h = 0 runs track them)
CASES = {
    "3d_field_bf16x6": (3, 0.2216544, 0.05, 6, 2, False),
    "3d_zero_field_bf16x6": (3, 0.2216544, 0.0, 6, 2, True),
    "2d_field_fp64": (2, 0.44, 0.02, 8, 0, False),
    "4d_field_tf32x3": (4, 0.15, 0.01, 3, 4, False),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_replayed_cycles_equal_the_uncaptured_run_bit_for_bit(pkg, case):
    d, beta, h, chi, prec, forget = CASES[case]
    cyc = 2 * d // np.gcd(2, d)           # lcm(2, d): the closed sequence
    warm = 2 * d + cyc                    # bond growth, then one uncaptured cycle
    axes = _axes(d, warm + 2 * cyc, d - 1)

    ref = pkg.Hotrg(d, beta, h, precision=prec, fp64_below=0.0)
    try:
        if forget:
            pkg.hotrg_set_parity(ref.ctx, None)
        want = []
        for i, a in enumerate(axes):
            ref.step(a, chi)
            if i + 1 in (warm + cyc, warm + 2 * cyc):
                want.append(_state(pkg, ref))
    finally:
        ref.close()

    g = pkg.Hotrg(d, beta, h, precision=prec, fp64_below=0.0)
    graph = None
    try:
        if forget:
            pkg.hotrg_set_parity(g.ctx, None)
        for a in axes[:warm]:
            g.step(a, chi)
        before = _state(pkg, g)
        graph = pkg.hotrg_graph_capture(g.ctx, axes[warm: warm + cyc], chi)
        # the capture runs nothing and leaves the context as it was
        after = _state(pkg, g)
        assert after[:4] == before[:4]
        np.testing.assert_array_equal(after[4], before[4])
        for k in range(2):
            pkg.hotrg_graph_launch(g.ctx, graph)
            got = _state(pkg, g)
            assert got[:4] == want[k][:4], (k, got[:4], want[k][:4])
            np.testing.assert_array_equal(got[4], want[k][4])
        # uncaptured steps continue from the replayed state
        g.step(axes[warm], chi)
        assert np.isfinite(g.free_energy()[0])
    finally:
        if graph is not None:
            pkg.hotrg_graph_free(graph)
        g.close()


def test_captures_that_cannot_be_replayed_are_refused(pkg):
    d, chi = 3, 6
    axes = _axes(d, 12, 2)
    g = pkg.Hotrg(d, 0.2216544, 0.0, precision=2, fp64_below=0.0)
    other = pkg.Hotrg(d, 0.2216544, 0.05, precision=2, fp64_below=0.0)
    graph = None
    try:
        for a in axes[:6]:
            g.step(a, chi)
        # known leg parities: the step waits for a host read-back
        with pytest.raises(pkg.HotrgError) as e:
            pkg.hotrg_graph_capture(g.ctx, axes[6:12], chi)
        assert e.value.status == ESTATE
        pkg.hotrg_set_parity(g.ctx, None)
        for a in axes[6:12]:
            g.step(a, chi)
        p0 = pkg.hotrg_observables(g.ctx)[2]
        lnz0 = g.free_energy()[0]
        # not closed: one step of a 3D run changes the slot order and the buffers
        with pytest.raises(pkg.HotrgError) as e:
            pkg.hotrg_graph_capture(g.ctx, axes[:1], chi)
        assert e.value.status == ESTATE
        # bond growth ahead: the steps would need larger buffers
        with pytest.raises(pkg.HotrgError) as e:
            pkg.hotrg_graph_capture(g.ctx, axes[:6], 2 * chi)
        assert e.value.status == ESTATE
        # the refused captures left the run as it was
        assert pkg.hotrg_observables(g.ctx)[2] == p0 and g.free_energy()[0] == lnz0
        graph = pkg.hotrg_graph_capture(g.ctx, axes[:6], chi)
        with pytest.raises(pkg.HotrgError) as e:     # another context's graph
            pkg.hotrg_graph_launch(other.ctx, graph)
        assert e.value.status == EINVAL
        g.step(axes[0], chi)
        with pytest.raises(pkg.HotrgError) as e:     # not at the start of its cycle
            pkg.hotrg_graph_launch(g.ctx, graph)
        assert e.value.status == ESTATE
    finally:
        if graph is not None:
            pkg.hotrg_graph_free(graph)
        g.close()
        other.close()
