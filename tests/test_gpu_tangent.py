"""GPU differentiation form (d/d beta in forward mode) through the C ABI against the
FP64 tangent oracle, finite differences of the GPU's own FP64 run, exact enumeration
and Onsager's internal energy."""

import numpy as np
import pytest

from oracle import hotrg_oracle as o
from oracle import hotrg_tangent as tg
from tests import exact_ising as ex

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch

    import paper_2110_03607_gb300 as p

    assert torch.cuda.is_available()
    p.load()
    return p


def _gpu_tangent_run(pkg, d, beta, h, chi, axes, z2=True, tensors_at=(), prec=0, fp64_below=None):
    g = pkg.Hotrg(d, beta, h, precision=prec, z2=z2, fp64_below=fp64_below)
    out, tens = [], {}
    try:
        pkg.hotrg_set_tangent(g.ctx, True)
        out.append(g.energy())
        for i, a in enumerate(axes):
            g.step(a, chi)
            lnz, _ = g.free_energy()
            dlnz, u, deg = g.energy()
            out.append((dlnz, u, deg, lnz))
            if i + 1 in tensors_at:
                tens[i + 1] = (pkg.hotrg_tensor(g.ctx), pkg.hotrg_tangent_tensor(g.ctx))
    finally:
        g.close()
    return out, tens


def _gpu_ln_z(pkg, d, beta, h, chi, axes):
    g = pkg.Hotrg(d, beta, h, precision=0)
    try:
        for a in axes:
            g.step(a, chi)
        return g.free_energy()[0]
    finally:
        g.close()


ORACLE_CASES = [
    (2, 0.35, 0.0, 8, 10),
    (2, 0.35, 0.0, 12, 12),
    (3, 0.21, 0.0, 6, 5),
    (2, 0.5, 0.05, 6, 10),
    (3, 0.2, 0.0, 4, 6),
    (3, 0.25, 0.1, 4, 5),
    (4, 0.15, 0.0, 3, 4),
]


@pytest.mark.parametrize("d,beta,h,chi,nsteps", ORACLE_CASES)
def test_energy_matches_oracle_every_step(pkg, d, beta, h, chi, nsteps):
    axes = o.cyclic_axes(d, nsteps)
    res, _ = _gpu_tangent_run(pkg, d, beta, h, chi, axes)
    r = tg.HotrgTangentRun(d, beta, h)
    assert res[0][0] == pytest.approx(r.dln_z, rel=1e-13)
    for i, a in enumerate(axes):
        rec = r.step(a, chi)
        dlnz, u, deg, lnz = res[i + 1]
        assert deg == rec.degenerate_pairs == 0
        assert abs(dlnz - rec.dln_z_per_site) <= 1e-10 * abs(rec.dln_z_per_site), (i, dlnz, rec.dln_z_per_site)
        assert u == -dlnz
        assert abs(lnz - rec.ln_z_per_site) <= 1e-12 * abs(rec.ln_z_per_site)


@pytest.mark.parametrize("d,beta,h,chi,nsteps", [(3, 0.25, 0.1, 4, 4), (2, 0.5, 0.05, 6, 5)])
def test_tangent_tensor_matches_oracle_elementwise(pkg, d, beta, h, chi, nsteps):
    axes = o.cyclic_axes(d, nsteps)
    _, tens = _gpu_tangent_run(pkg, d, beta, h, chi, axes, tensors_at=range(1, nsteps + 1))
    r = tg.HotrgTangentRun(d, beta, h)
    for i, a in enumerate(axes):
        r.step(a, chi)
        t_gpu, dt_gpu = tens[i + 1]
        assert t_gpu.shape == r.t.shape and dt_gpu.shape == r.dt.shape
        np.testing.assert_allclose(t_gpu, r.t, rtol=0, atol=1e-12 * np.abs(r.t).max())
        np.testing.assert_allclose(dt_gpu, r.dt, rtol=0, atol=1e-10 * np.abs(r.dt).max())


def test_z2_setting_does_not_change_the_derivative(pkg):
    # block-form eigen-solver (z2 on) or dense (off): the same derivative up to rounding
    axes = o.cyclic_axes(3, 5)
    a, _ = _gpu_tangent_run(pkg, 3, 0.22, 0.0, 6, axes, z2=True)
    b, _ = _gpu_tangent_run(pkg, 3, 0.22, 0.0, 6, axes, z2=False)
    for x, y in zip(a[1:], b[1:]):
        assert abs(x[0] - y[0]) <= 1e-11 * abs(y[0])


# Near beta_c, ln Z of a truncated run is not smooth on the scale of 1e-5 in beta for
# every chi (2D chi = 16, beta = 0.42: the oracle's own central differences with steps
# 1e-4, 1e-5, 1e-6 scatter by 1e-3); the cases here are ones where they agree.
@pytest.mark.parametrize("d,beta,h,chi,nsteps", [(3, 0.22, 0.0, 8, 9), (2, 0.42, 0.0, 12, 16),
                                                  (4, 0.16, 0.02, 4, 6)])
def test_energy_matches_central_difference_of_the_gpu_run(pkg, d, beta, h, chi, nsteps):
    axes = o.cyclic_axes(d, nsteps)
    res, _ = _gpu_tangent_run(pkg, d, beta, h, chi, axes)
    db = 1e-5
    fd = (_gpu_ln_z(pkg, d, beta + db, h, chi, axes) - _gpu_ln_z(pkg, d, beta - db, h, chi, axes)) / (2 * db)
    dlnz, _, deg, _ = res[-1]
    assert deg == 0
    assert abs(dlnz - fd) <= 1e-7 * abs(fd), (dlnz, fd)


# Steps whose kept and discarded eigenvalues are exactly degenerate (3D chi = 8,
# beta = 0.22, steps 2-3: gaps of 5e-18 lambda_1) keep an arbitrary vector of the
# degenerate pair; the FP64 and split runs keep different ones there and their
# derivatives then differ by up to 4e-4.  Such small steps run in FP64 under the
# default threshold, as in the 3D case below.
@pytest.mark.parametrize("d,beta,h,chi,nsteps,fp64_below,gate", [
    (3, 0.2216544, 0.0, 12, 10, None, 1e-6),  # growth steps in FP64, the rest split
    (2, 0.35, 0.02, 12, 12, 0.0, 1e-6),       # every step split
])
def test_split_bf16_derivative_matches_fp64(pkg, d, beta, h, chi, nsteps, fp64_below, gate):
    # the contraction of the derivative in split BF16 (6 terms, FP32 accumulation) against FP64
    axes = o.cyclic_axes(d, nsteps)
    ref, _ = _gpu_tangent_run(pkg, d, beta, h, chi, axes, prec=0)
    got, _ = _gpu_tangent_run(pkg, d, beta, h, chi, axes, prec=2, fp64_below=fp64_below)
    errs = [abs(x[0] - y[0]) / abs(y[0]) for x, y in zip(got[1:], ref[1:])]
    print("split-BF16 derivative, relative errors by step:", ["%.1e" % e for e in errs])
    assert max(errs) <= gate, errs
    lnz_errs = [abs(x[3] - y[3]) / abs(y[3]) for x, y in zip(got[1:], ref[1:])]
    assert max(lnz_errs) <= 5e-7, lnz_errs   # the forward gate of forced split steps


@pytest.mark.parametrize("d,nsteps,chi,beta,h", [(2, 4, 16, 0.3, 0.1), (3, 3, 16, 0.25, 0.05)])
def test_untruncated_energy_equals_brute_force(pkg, d, nsteps, chi, beta, h):
    axes = o.cyclic_axes(d, nsteps, first=d - 1)
    res, _ = _gpu_tangent_run(pkg, d, beta, h, chi, axes)
    assert res[0][1] == pytest.approx(ex.brute_force_energy((1,) * d, beta, h), rel=1e-13)
    for i in range(nsteps):
        exact = ex.brute_force_energy(ex.lattice_after(d, axes[: i + 1]), beta, h)
        assert res[i + 1][1] == pytest.approx(exact, rel=1e-11, abs=1e-13), i


@pytest.mark.parametrize("beta,chi,gate", [(0.3, 16, 1e-7), (0.5, 16, 1.5e-6), (0.4, 16, 6e-6)])
def test_energy_against_onsager(pkg, beta, chi, gate):
    axes = o.cyclic_axes(2, 24)
    res, _ = _gpu_tangent_run(pkg, 2, beta, 0.0, chi, axes)
    _, u, deg, _ = res[-1]
    exact = ex.onsager_energy_per_site(beta)
    assert abs(u - exact) / abs(exact) <= gate, (u, exact, deg)


def test_batch_of_tangent_contexts_equals_separate_runs(pkg):
    # the scan path: contexts carrying the derivative, stepped together on their own streams
    import torch

    insts = [(3, 0.215, 0.0, 6), (3, 0.22, 0.01, 8), (2, 0.4, 0.0, 10)]
    axes = [0, 1, 2, 0, 1, 2]
    alone = []
    for d, b, h, chi in insts:
        res, _ = _gpu_tangent_run(pkg, d, b, h, chi, [a % d for a in axes], prec=2, fp64_below=0.0)
        alone.append(res[-1])
    streams = [torch.cuda.Stream() for _ in insts]
    ctxs = []
    try:
        for (d, b, h, chi), st in zip(insts, streams):
            c = pkg.hotrg_init_ising(d, b, h)
            pkg.hotrg_set_precision(c, 2)
            pkg.hotrg_set_fp64_threshold(c, 0.0)
            pkg.hotrg_set_stream(c, st.cuda_stream)
            pkg.hotrg_set_tangent(c, True)
            ctxs.append(c)
        for a in axes:
            pkg.hotrg_step_batch(ctxs, [a % d for d, _, _, _ in insts], [x[3] for x in insts], 3)
        for c, ref in zip(ctxs, alone):
            dlnz, u, deg = pkg.hotrg_energy(c)
            assert (dlnz, deg) == (ref[0], ref[2])
    finally:
        for c in ctxs:
            pkg.hotrg_free(c)


def test_allocator_switch_keeps_the_derivative(pkg):
    # hotrg_set_allocator drops the workspaces but keeps T, dT and both run states
    import torch

    axes = o.cyclic_axes(3, 5)
    ref, _ = _gpu_tangent_run(pkg, 3, 0.22, 0.0, 6, axes)
    c = pkg.hotrg_init_ising(3, 0.22, 0.0)
    g = pkg.Hotrg.__new__(pkg.Hotrg)   # owning handle around the raw context (frees it once)
    g.ctx, g._cb = c, None
    try:
        pkg.hotrg_set_precision(c, 0)
        pkg.hotrg_set_stream(c, torch.cuda.current_stream().cuda_stream)
        pkg.hotrg_set_tangent(c, True)
        for a in axes[:2]:
            pkg.hotrg_step(c, a, 6)
        g.use_torch()                      # switch to the torch allocator mid-run
        for a in axes[2:]:
            pkg.hotrg_step(c, a, 6)
        assert pkg.hotrg_energy(c)[0] == ref[-1][0]
    finally:
        g.close()


def test_bad_arguments(pkg):
    g = pkg.Hotrg(2, 0.3, 0.0)
    try:
        with pytest.raises(pkg.HotrgError):
            g.energy()                          # not carried
        g.step(0, 4)
        with pytest.raises(pkg.HotrgError):
            pkg.hotrg_set_tangent(g.ctx, True)  # steps already taken
    finally:
        g.close()
    g = pkg.Hotrg(2, 0.0, 0.0)
    try:
        with pytest.raises(pkg.HotrgError):
            pkg.hotrg_set_tangent(g.ctx, True)  # beta = 0
    finally:
        g.close()
    t = o.initial_tensor(2, 0.3, 0.0)
    g = pkg.Hotrg(2, 0.3, tensor=np.ascontiguousarray(t), chis=[2, 2])
    try:
        with pytest.raises(pkg.HotrgError):
            pkg.hotrg_set_tangent(g.ctx, True)  # not an Ising context
    finally:
        g.close()


def test_autograd_function_gives_the_tangent_oracle_gradient(pkg):
    # torch.autograd on ln Z/V (the C ABI's forward-mode tangent in the backward pass)
    # against the tangent oracle, step by step, and against the plain central difference
    # of the forward values
    import torch

    from paper_2110_03607_gb300 import autograd as ag

    d, beta, h, chi = 3, 0.22, 0.0, 4
    axes = o.cyclic_axes(d, 6, first=2)
    bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    lnz = ag.ln_z_per_site(bt, d, h, chi, axes)
    tr = tg.HotrgTangentRun(d, beta, h)
    recs = [tr.step(a, chi) for a in axes]
    for p in range(len(axes)):
        (g,) = torch.autograd.grad(lnz[p], bt, retain_graph=True)
        want = recs[p].dln_z_per_site
        assert abs(float(g) - want) <= 1e-10 * abs(want), (p, float(g), want)
    # a weighted sum: the vector-Jacobian product
    w = torch.linspace(0.5, 2.0, len(axes), dtype=torch.float64)
    (gw,) = torch.autograd.grad((w * lnz).sum(), bt)
    want = sum(float(w[p]) * recs[p].dln_z_per_site for p in range(len(axes)))
    assert abs(float(gw) - want) <= 1e-10 * abs(want)
    # central difference of the forward values (beta +- 1e-5)
    db = 1e-5
    with torch.no_grad():
        up = ag.ln_z_per_site(torch.tensor(beta + db, dtype=torch.float64), d, h, chi, axes)[-1]
        dn = ag.ln_z_per_site(torch.tensor(beta - db, dtype=torch.float64), d, h, chi, axes)[-1]
    fd = float(up - dn) / (2 * db)
    assert abs(ag.energy_per_site(beta, d, h, chi, axes) + fd) <= 1e-7 * abs(fd)
