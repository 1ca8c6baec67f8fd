"""The default multi-GPU path of bench.py runs replicas (independent runs, no collective on
the data path): the timing reduction and the whole-job rate, on two gloo ranks (CPU); and
the argument check of its sharded form (--shard, one run split over NCCL ranks)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank "ran" 10 steps in a different time; the job is as slow as the slowest
        ms = 1000.0 + 250.0 * rank
        slowest = bench.max_over_ranks(ms, dist, "cpu")
        out[rank] = (slowest, bench.whole_job_rate(10, world, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank_and_the_aggregate_rate():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        slowest, rate = res[r]
        assert slowest == 1250.0
        assert rate == pytest.approx(2 * 10 / 1.25)


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.whole_job_rate(24, 1, 2000.0) == pytest.approx(12.0)


def test_shard_flag_refuses_workloads_it_does_not_time():
    # bench.py --shard times the c'-slice shard of one run (NCCL); the batching and
    # differentiation workloads have no sharded form, and the refusal comes from the
    # argument check before any device is touched
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for wl in ("batch3d_mixed", "energy3d_chi12"):
        r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--shard", "--workload", wl],
                           capture_output=True, text=True, timeout=120)
        assert r.returncode == 2, r.stderr
        assert "--shard" in r.stderr
