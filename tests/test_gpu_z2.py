"""Z2 block form of the new-tensor contraction (zero field) against the oracle,
the dense form, and the exact zero pattern of the Ising tensor."""

import numpy as np
import pytest

from oracle import hotrg_oracle as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch

    import paper_2110_03607_gb300 as p

    assert torch.cuda.is_available()
    p.load()
    return p


def _odd_mask(shape, parity, d):
    # parity: per axis a 0/1 vector; both legs of an axis share it
    tot = np.zeros(shape, dtype=np.int64)
    for k in range(d):
        for side in (0, 1):
            sh = [1] * (2 * d)
            sh[2 * k + side] = shape[2 * k + side]
            tot = tot + np.asarray(parity[k]).reshape(sh)
    return (tot % 2) == 1


def _split_parity(flat, dims):
    out, off = [], 0
    for n in dims:
        out.append(np.array(flat[off:off + n]))
        off += n
    return out


def _oracle_parities(d, legs_per_step):
    """Leg parities after each oracle step, from the support of the isometry columns."""
    parity = [np.array([0, 1])] * d
    hist = []
    for legs in legs_per_step:
        new = list(parity)
        for leg in legs:
            pj = parity[leg.axis]
            row = ((pj[None, :] + pj[:, None]) % 2).reshape(-1)   # row hat + check * chi
            cols = []
            for k in range(leg.u.shape[1]):
                ps = set(row[np.abs(leg.u[:, k]) > 0].tolist())
                assert len(ps) == 1
                cols.append(ps.pop())
            new[leg.axis] = np.array(cols)
        parity = new
        hist.append(parity)
    return hist


@pytest.mark.parametrize("d,chi,nsteps,beta", [
    (2, 8, 10, 0.4406868),
    (3, 6, 6, 0.2216544),
    (4, 3, 5, 0.15),
])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (2, 5e-7)])
def test_z2_blocks_match_oracle(pkg, d, chi, nsteps, beta, prec, tol):
    axes = o.cyclic_axes(d, nsteps)
    g = pkg.Hotrg(d, beta, 0.0, precision=prec, fp64_below=0.0, z2=True)
    run = o.HotrgRun(d, beta, 0.0)
    try:
        for a in axes:
            g.step(a, chi)
            rec = run.step(a, chi)
            lnz, _ = g.free_energy()
            assert abs(lnz - rec.ln_z_per_site) / abs(rec.ln_z_per_site) <= tol, (rec.step, lnz)
            dense, done, used = pkg.hotrg_bottleneck_flops(g.ctx)
            assert used
            # two blocks of (R/2)^2 (N/2) each when the parities split evenly
            assert 0.0 < done <= 0.5 * dense
    finally:
        g.close()


@pytest.mark.parametrize("d,chi,nsteps", [(2, 8, 8), (3, 5, 6), (4, 3, 4)])
def test_z2_fp64_agrees_with_the_dense_form(pkg, d, chi, nsteps):
    # the blocks drop only products with an exact-zero factor; the Grams' split-K
    # partial sums are grouped differently, so the two FP64 runs agree to rounding
    axes = o.cyclic_axes(d, nsteps)
    ga = pkg.Hotrg(d, 0.3, 0.0, precision=pkg.PREC_FP64, z2=True)
    gb = pkg.Hotrg(d, 0.3, 0.0, precision=pkg.PREC_FP64, z2=False)
    try:
        for a in axes:
            ga.step(a, chi)
            gb.step(a, chi)
            assert pkg.hotrg_bottleneck_flops(ga.ctx)[2]
            assert not pkg.hotrg_bottleneck_flops(gb.ctx)[2]
            la, lb = ga.free_energy()[0], gb.free_energy()[0]
            assert abs(la - lb) <= 1e-14 * abs(lb)
            xa = pkg.hotrg_observables(ga.ctx)[1]
            xb = pkg.hotrg_observables(gb.ctx)[1]
            assert abs(xa - xb) <= 1e-11
            # the gauge-fixed tensors themselves, element by element, to the FP64 parity
            # gate of T' (the rounding of the regrouped Gram sums moves the eigenvectors
            # by ~1e-11 after 8 steps)
            ta = pkg.hotrg_tensor(ga.ctx)
            tb = pkg.hotrg_tensor(gb.ctx)
            assert ta.shape == tb.shape
            np.testing.assert_allclose(ta, tb, rtol=0, atol=1e-10 * np.abs(tb).max())
    finally:
        ga.close()
        gb.close()


@pytest.mark.parametrize("z2", [True, False])
@pytest.mark.parametrize("prec", [0, 2])
def test_odd_parity_elements_are_exactly_zero(pkg, z2, prec):
    d, chi = 3, 6
    g = pkg.Hotrg(d, 0.2216544, 0.0, precision=prec, fp64_below=0.0, z2=z2)
    try:
        for a in o.cyclic_axes(d, 6):
            g.step(a, chi)
            t = pkg.hotrg_tensor(g.ctx)
            dims = pkg.hotrg_bond_dims(g.ctx)[:d]
            par = pkg.hotrg_leg_parity(g.ctx)
            assert par is not None and len(par) == sum(dims)
            odd = _odd_mask(t.shape, _split_parity(par, dims), d)
            assert odd.any() and (~odd).any()
            assert np.count_nonzero(t[odd]) == 0
    finally:
        g.close()


def test_leg_parities_match_the_oracle_isometries(pkg):
    d, chi = 3, 6
    axes = o.cyclic_axes(d, 5)
    g = pkg.Hotrg(d, 0.2216544, 0.0, precision=pkg.PREC_FP64)
    run = o.HotrgRun(d, 0.2216544, 0.0)
    try:
        legs = []
        for a in axes:
            g.step(a, chi)
            legs.append(run.step(a, chi).legs)
        want = _oracle_parities(d, legs)[-1]
        dims = pkg.hotrg_bond_dims(g.ctx)[:d]
        got = _split_parity(pkg.hotrg_leg_parity(g.ctx), dims)
        for k in range(d):
            assert np.array_equal(got[k], want[k]), k
    finally:
        g.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (2, 5e-7)])
@pytest.mark.parametrize("d,chi,nsteps", [(3, 5, 6), (4, 3, 5), (2, 6, 8)])
def test_z2_with_n1_sub_slices_matches_oracle(pkg, prec, tol, d, chi, nsteps):
    # a 1-byte budget: one n'_1 value per sub-slice, each with its own column maps
    beta = 0.25
    axes = o.cyclic_axes(d, nsteps)
    g = pkg.Hotrg(d, beta, 0.0, precision=prec, fp64_below=0.0, z2=True)
    run = o.HotrgRun(d, beta, 0.0)
    try:
        pkg.hotrg_set_slice_budget(g.ctx, 1.0)
        for a in axes:
            g.step(a, chi)
            rec = run.step(a, chi)
            lnz, _ = g.free_energy()
            assert pkg.hotrg_bottleneck_flops(g.ctx)[2]
            assert abs(lnz - rec.ln_z_per_site) / abs(rec.ln_z_per_site) <= tol, (rec.step, lnz)
    finally:
        g.close()


def test_nonzero_field_has_no_parities(pkg):
    g = pkg.Hotrg(3, 0.25, 0.05, precision=pkg.PREC_BF16X6, fp64_below=0.0)
    try:
        assert pkg.hotrg_leg_parity(g.ctx) is None
        g.step(2, 4)
        assert not pkg.hotrg_bottleneck_flops(g.ctx)[2]
        assert pkg.hotrg_leg_parity(g.ctx) is None
    finally:
        g.close()


def test_chi_one_leaves_only_even_blocks(pkg):
    # chi = 1 keeps the single dominant (even) state: the odd blocks are empty
    for prec in (0, 2):
        g = pkg.Hotrg(3, 0.2, 0.0, precision=prec, fp64_below=0.0)
        run = o.HotrgRun(3, 0.2, 0.0)
        try:
            for a in o.cyclic_axes(3, 4):
                g.step(a, 1)
                rec = run.step(a, 1)
                lnz, _ = g.free_energy()
                assert abs(lnz - rec.ln_z_per_site) / abs(rec.ln_z_per_site) <= 1e-7
        finally:
            g.close()


def test_set_parity_checks_the_tensor_and_enables_blocks(pkg):
    beta, chi = 0.25, 5
    run = o.HotrgRun(3, beta, 0.0)
    legs = [run.step(2, chi).legs, run.step(0, chi).legs]
    par = _oracle_parities(3, legs)[-1]
    t_in = run.t.copy()
    chis = [t_in.shape[2 * k] for k in range(3)]
    flat = [int(x) for k in range(3) for x in par[k]]
    ctx = pkg.hotrg_init_tensor(3, chis, t_in, beta)
    try:
        assert pkg.hotrg_leg_parity(ctx) is None
        bad = list(flat)
        bad[0] ^= 1
        with pytest.raises(pkg.HotrgError):
            pkg.hotrg_set_parity(ctx, bad)
        with pytest.raises(pkg.HotrgError):
            pkg.hotrg_set_parity(ctx, [2] + flat[1:])
        assert pkg.hotrg_leg_parity(ctx) is None
        pkg.hotrg_set_parity(ctx, flat)
        assert pkg.hotrg_leg_parity(ctx) == flat
        pkg.hotrg_set_precision(ctx, pkg.PREC_FP64)
        pkg.hotrg_step(ctx, 1, chi)
        assert pkg.hotrg_bottleneck_flops(ctx)[2]
        run.step(1, chi)
        t_gpu = pkg.hotrg_tensor(ctx)
        np.testing.assert_allclose(t_gpu, run.t, rtol=0, atol=1e-9 * np.abs(run.t).max())
    finally:
        pkg.hotrg_free(ctx)


def test_ising3d_chi16_sampled_new_tensor_elements_z2(pkg):
    # as the dense full-size test: the oracle's tensor after steps z, x, y (bonds
    # 16, 16, 16), with its leg parities declared; one full-size step along z
    # (split-BF16, Z2 blocks); sampled (c', n') slabs of T_new from the oracle
    run = o.HotrgRun(3, 0.2216544, 0.0)
    legs = [run.step(a, 16).legs for a in (2, 0, 1)]
    par = _oracle_parities(3, legs)[-1]
    t_in = run.t
    ctx = pkg.hotrg_init_tensor(3, [16, 16, 16], t_in, 0.2216544)
    try:
        pkg.hotrg_set_parity(ctx, [int(x) for k in range(3) for x in par[k]])
        pkg.hotrg_set_precision(ctx, pkg.PREC_BF16X6)
        pkg.hotrg_step(ctx, 2, 16)
        dense, done, used = pkg.hotrg_bottleneck_flops(ctx)
        assert used and done <= 0.26 * dense
        tr_gpu, _, _ = pkg.hotrg_observables(ctx)
        t_gpu = pkg.hotrg_tensor(ctx) * tr_gpu
        tp = o.to_paper_order(t_in, 2)
        nxt = o.next_axes(3, 2)
        olegs = [o.choose_isometry(tp, j, 16, nxt[j - 1]) for j in (1, 2)]
        tgpu_p = o.to_paper_order(t_gpu, 2)
        that = o.hat_matrix(tp)
        rng = np.random.default_rng(11)
        for _ in range(6):
            c0p = int(rng.integers(16))
            npr = (int(rng.integers(16)), int(rng.integers(16)))
            slab = o.new_tensor_slab(tp, [leg.u for leg in olegs], c0p, npr, that)
            got = np.moveaxis(tgpu_p[:, :, npr[1], npr[0], :, c0p], -1, 0)
            scale = np.abs(slab).max()
            np.testing.assert_allclose(got, slab, rtol=0, atol=2e-6 * scale)
    finally:
        pkg.hotrg_free(ctx)


def test_unbalanced_parities_match_the_dense_form(pkg):
    # 3D chi=12 at beta = 0.20 keeps mostly even states after a few steps: the padded
    # eigen blocks then outgrow the dense matrices (one parity holds more than 0.707 of
    # a leg's composite states).  The Z2 run must agree with the dense run (FP64 form).
    d, chi, nsteps = 3, 12, 8
    ga = pkg.Hotrg(d, 0.20, 0.0, precision=pkg.PREC_FP64, z2=True)
    gb = pkg.Hotrg(d, 0.20, 0.0, precision=pkg.PREC_FP64, z2=False)
    worst = 0.0
    try:
        for a in o.cyclic_axes(d, nsteps):
            ga.step(a, chi)
            gb.step(a, chi)
            la, lb = ga.free_energy()[0], gb.free_energy()[0]
            assert abs(la - lb) <= 1e-13 * abs(lb)
            dims = pkg.hotrg_bond_dims(ga.ctx)[:d]
            for p in _split_parity(pkg.hotrg_leg_parity(ga.ctx), dims):
                e = int((p == 0).sum())
                # share of the even composite (hat, check) states of this leg
                worst = max(worst, (e * e + (len(p) - e) ** 2) / len(p) ** 2)
        assert worst > 0.75, worst   # the padded case was exercised
    finally:
        ga.close()
        gb.close()
