"""Batching form: hotrg_step_batch drives independent contexts concurrently; every
instance must come out exactly as when stepped alone, and match the oracle."""

import pytest

from oracle import hotrg_oracle as o

pytestmark = pytest.mark.gpu

# (d, beta, h, chi): mixed dimensions, fields and bond dimensions
INSTANCES = [(3, 0.20, 0.0, 4), (3, 0.22, 0.01, 5), (3, 0.24, 0.0, 6), (3, 0.21, 0.01, 3),
             (2, 0.44, 0.0, 8), (4, 0.15, 0.0, 3)]


@pytest.fixture(scope="module")
def pkg():
    import torch

    import paper_2110_03607_gb300 as p

    assert torch.cuda.is_available()
    p.load()
    return p


def _contexts(pkg, streams, prec):
    ctxs = []
    for (d, beta, h, _), st in zip(INSTANCES, streams):
        c = pkg.hotrg_init_ising(d, beta, h)
        pkg.hotrg_set_precision(c, prec)
        pkg.hotrg_set_fp64_threshold(c, 0.0)
        pkg.hotrg_set_stream(c, st.cuda_stream if st is not None else None)
        ctxs.append(c)
    return ctxs


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("nthreads", [1, 4, 0])
def test_batch_equals_separate_runs_bit_for_bit(pkg, prec, nthreads):
    import torch

    nsteps = 5
    streams = [torch.cuda.Stream() for _ in INSTANCES]
    batch = _contexts(pkg, streams, prec)
    alone = _contexts(pkg, [None] * len(INSTANCES), prec)
    try:
        for s in range(nsteps):
            axes = [(s + d - 1) % d for d, _, _, _ in INSTANCES]
            chis = [x[3] for x in INSTANCES]
            st = pkg.hotrg_step_batch(batch, axes, chis, nthreads)
            assert st == [0] * len(INSTANCES)
            for c, a, chi in zip(alone, axes, chis):
                pkg.hotrg_step(c, a, chi)
            for cb, ca in zip(batch, alone):
                assert pkg.hotrg_free_energy(cb) == pkg.hotrg_free_energy(ca)
                assert pkg.hotrg_observables(cb) == pkg.hotrg_observables(ca)
    finally:
        for c in batch + alone:
            pkg.hotrg_free(c)


def test_batch_instances_match_the_oracle(pkg):
    import torch

    nsteps = 4
    streams = [torch.cuda.Stream() for _ in INSTANCES]
    ctxs = _contexts(pkg, streams, pkg.PREC_FP64)
    runs = [o.HotrgRun(d, beta, h) for d, beta, h, _ in INSTANCES]
    try:
        for s in range(nsteps):
            axes = [(s + d - 1) % d for d, _, _, _ in INSTANCES]
            pkg.hotrg_step_batch(ctxs, axes, [x[3] for x in INSTANCES])
            for c, run, a, inst in zip(ctxs, runs, axes, INSTANCES):
                rec = run.step(a, inst[3])
                lnz = pkg.hotrg_free_energy(c)[0]
                assert abs(lnz - rec.ln_z_per_site) <= 1e-12 * abs(rec.ln_z_per_site), (inst, s)
    finally:
        for c in ctxs:
            pkg.hotrg_free(c)


def test_batch_rejects_bad_arguments(pkg):
    c = pkg.hotrg_init_ising(2, 0.3, 0.0)
    try:
        with pytest.raises(pkg.HotrgError):
            pkg.hotrg_step_batch([c, c], [0, 0], [4, 4])     # the same context twice
        st = None
        with pytest.raises(pkg.HotrgError):
            pkg.hotrg_step_batch([c], [5], [4])              # axis out of range
        del st
    finally:
        pkg.hotrg_free(c)
