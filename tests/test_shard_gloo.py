"""Host logic of the c'-slice shard (paper_2110_03607_gb300/shard.py) on two gloo ranks
on the CPU: the slice partition, the sum of the partial Grams, and the order of the
gathered slices.  The library calls are replaced by fakes that record what they get,
so no GPU is needed; the GPU test (test_gpu_shard.py) runs the real kernels."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2110_03607_gb300 import shard


def test_slice_ranges_cover_every_slice_once():
    for chi_c in (1, 2, 5, 16, 17):
        for world in (1, 2, 3, 4, 8):
            seen = []
            for r in range(world):
                lo, hi = shard.slice_range(chi_c, r, world)
                assert 0 <= lo <= hi <= chi_c
                seen.extend(range(lo, hi))
            assert seen == list(range(chi_c))
            sizes = [hi - lo for lo, hi in (shard.slice_range(chi_c, r, world) for r in range(world))]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


N_GRAMS, CHI_C, PER_SLICE = 7, 5, 3


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_2110_03607_gb300 import binding as b

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seen = {}

    # fakes with the calling convention of the real binding
    b.shard_sizes = lambda ctx, axis, chi: (N_GRAMS, CHI_C, PER_SLICE)

    def env(ctx, axis, chi, part, nparts, out=None):
        assert (part, nparts) == (rank, world)
        out.copy_(torch.arange(N_GRAMS, dtype=torch.float64) * 10.0 ** rank)
        return out

    def iso(ctx, axis, chi, grams):
        seen["grams"] = grams.clone().numpy()

    def contract(ctx, axis, chi, lo, hi, out=None):
        assert (lo, hi) == shard.slice_range(CHI_C, rank, world)
        vals = [100.0 * sl + e for sl in range(lo, hi) for e in range(PER_SLICE)]
        out.copy_(torch.tensor(vals, dtype=torch.float64))
        return out

    def finish(ctx, axis, chi, slices):
        seen["slices"] = slices.clone().numpy()

    b.hotrg_shard_env, b.hotrg_shard_isometries = env, iso
    b.hotrg_shard_contract, b.hotrg_shard_finish = contract, finish
    shard.step_sharded(None, 0, 4)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), **seen)
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_grams_and_gather_slices_in_order(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    want_grams = sum(np.arange(N_GRAMS) * 10.0 ** r for r in range(world))
    want_slices = np.array([100.0 * sl + e for sl in range(CHI_C) for e in range(PER_SLICE)])
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npz")
        np.testing.assert_array_equal(got["grams"], want_grams)
        np.testing.assert_array_equal(got["slices"], want_slices)
