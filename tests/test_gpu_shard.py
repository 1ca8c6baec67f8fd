"""c'-slice shard of a step (hotrg_shard_*) on two processes that share cuda:0, with
gloo collectives between them, against the same steps taken by one process with
hotrg_step.  No kernel of one rank waits on the other: the ranks meet only in the
host-side collectives.

* slices only: every rank computes the whole environment Grams (no reduction), so
  both take the same isometries as hotrg_step; the contraction is split by c'-slices
  and gathered -- the new tensor must equal hotrg_step's bit for bit;
* the full shard: each rank sums its part of the Grams' summed index and the parts
  are summed over the ranks -- equal to hotrg_step up to the grouping of that sum.
"""

import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# d, beta, h, chi, steps, precision (0 FP64, 2 BF16X6)
CASES = {
    "3d_fp64": (3, 0.2216544, 0.0, 6, 6, 0),
    "3d_bf16x6": (3, 0.2216544, 0.0, 6, 6, 2),
    "2d_field_fp64": (2, 0.4, 0.05, 8, 8, 0),
    "4d_fp64": (4, 0.15, 0.0, 3, 5, 0),
}


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _axes(d, n):
    return [(d - 1 + s) % d for s in range(n)]


def _rank(rank, world, port, out_dir, case, reduce_grams):
    import torch
    import torch.distributed as dist

    import paper_2110_03607_gb300 as pkg
    from paper_2110_03607_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    d, beta, h, chi, nsteps, prec = CASES[case]
    g = pkg.Hotrg(d, beta, h, precision=prec, fp64_below=0.0)
    lnz = []
    for a in _axes(d, nsteps):
        if reduce_grams:
            shard.step_sharded(g.ctx, a, chi)
        else:
            # every rank takes the whole Grams: same isometries as one process
            grams = pkg.hotrg_shard_env(g.ctx, a, chi, 0, 1)
            pkg.hotrg_shard_isometries(g.ctx, a, chi, grams)
            _, chi_c, per = pkg.shard_sizes(g.ctx, a, chi)
            lo, hi = shard.slice_range(chi_c, rank, world)
            mine = torch.from_numpy(pkg.hotrg_shard_contract(g.ctx, a, chi, lo, hi))
            sizes = [shard.slice_range(chi_c, r, world) for r in range(world)]
            pad = max(b - a_ for a_, b in sizes) * per
            buf = torch.zeros(pad, dtype=torch.float64)
            buf[: mine.numel()] = mine
            parts = [torch.empty_like(buf) for _ in range(world)]
            dist.all_gather(parts, buf)
            full = torch.cat([p[: (b - a_) * per] for p, (a_, b) in zip(parts, sizes)])
            pkg.hotrg_shard_finish(g.ctx, a, chi, full.numpy())
        lnz.append(g.free_energy()[0])
    t = pkg.hotrg_tensor(g.ctx)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), lnz=np.array(lnz), t=t)
    g.close()
    dist.destroy_process_group()


def _reference(case):
    import paper_2110_03607_gb300 as pkg

    d, beta, h, chi, nsteps, prec = CASES[case]
    g = pkg.Hotrg(d, beta, h, precision=prec, fp64_below=0.0)
    lnz = []
    try:
        for a in _axes(d, nsteps):
            g.step(a, chi)
            lnz.append(g.free_energy()[0])
        return np.array(lnz), pkg.hotrg_tensor(g.ctx)
    finally:
        g.close()


def _run(tmp_path, case, reduce_grams, world=2):
    import torch.multiprocessing as mp

    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path), case, reduce_grams), nprocs=world, join=True)
    return [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]


@pytest.mark.parametrize("case", sorted(CASES))
def test_slice_partition_equals_one_process_bit_for_bit(tmp_path, case):
    ranks = _run(tmp_path, case, reduce_grams=False)
    lnz, t = _reference(case)
    for r in ranks:
        np.testing.assert_array_equal(r["lnz"], lnz)
        np.testing.assert_array_equal(r["t"], t)


@pytest.mark.parametrize("case", sorted(CASES))
def test_sharded_step_with_gram_reduction_matches_one_process(tmp_path, case):
    ranks = _run(tmp_path, case, reduce_grams=True)
    lnz, t = _reference(case)
    prec = CASES[case][5]
    tol_z, tol_t = (1e-13, 1e-10) if prec == 0 else (1e-10, 1e-8)
    # the ranks sum the same reduced Grams: they agree with each other exactly
    np.testing.assert_array_equal(ranks[0]["lnz"], ranks[1]["lnz"])
    np.testing.assert_array_equal(ranks[0]["t"], ranks[1]["t"])
    np.testing.assert_allclose(ranks[0]["lnz"], lnz, rtol=tol_z, atol=0)
    np.testing.assert_allclose(ranks[0]["t"], t, rtol=0, atol=tol_t * np.abs(t).max())


def test_shard_calls_out_of_order_are_refused():
    import paper_2110_03607_gb300 as pkg

    g = pkg.Hotrg(3, 0.22, 0.0, precision=0)
    try:
        with pytest.raises(pkg.HotrgError):      # no isometries installed yet
            pkg.hotrg_shard_contract(g.ctx, 2, 4, 0, 1)
        grams = pkg.hotrg_shard_env(g.ctx, 2, 4, 0, 1)
        with pytest.raises(pkg.HotrgError):      # wrong Gram count
            pkg.hotrg_shard_isometries(g.ctx, 2, 4, grams[:-1])
        with pytest.raises(pkg.HotrgError):      # part outside [0, nparts)
            pkg.hotrg_shard_env(g.ctx, 2, 4, 2, 2)
        pkg.hotrg_shard_isometries(g.ctx, 2, 4, grams)
        with pytest.raises(pkg.HotrgError):      # another axis than the installed isometries'
            pkg.hotrg_shard_contract(g.ctx, 1, 4, 0, 1)
        with pytest.raises(pkg.HotrgError):      # empty slice range
            pkg.hotrg_shard_contract(g.ctx, 2, 4, 1, 1)
        slices = pkg.hotrg_shard_contract(g.ctx, 2, 4, 0, 2)
        pkg.hotrg_shard_finish(g.ctx, 2, 4, slices)
        assert pkg.hotrg_observables(g.ctx)[2] == 1
    finally:
        g.close()
