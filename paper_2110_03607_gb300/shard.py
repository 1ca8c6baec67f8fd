"""c'-slice shard of one coarse-graining step over the ranks of a process group.

Every rank holds a context with the same local tensor (the paper replicates T
over its processes, Secs. 3.2 and 4.2.3-4.2.4).  One step is four calls of the
C ABI with two collectives between them:

  1. hotrg_shard_env          this rank's share of the environment Grams
  2. all_reduce (sum)         the Grams of the whole summed index
  3. hotrg_shard_isometries   A, eigen-solver, choice and truncation (same on every rank)
  4. hotrg_shard_contract     the new tensor's c'-slices of this rank
  5. all_gather               every slice, in c' order
  6. hotrg_shard_finish       install the new tensor, trace / ln Z / normalisation

This module only moves buffers between the library and torch.distributed; every
step of the arithmetic runs in libhotrg.so.  With the NCCL backend the buffers
are device tensors, otherwise host tensors.
"""

from __future__ import annotations

from . import binding as _b


def slice_range(chi_c: int, rank: int, world: int):
    """The c'-slices [lo, hi) of `rank`: contiguous, sizes differing by at most one."""
    return chi_c * rank // world, chi_c * (rank + 1) // world


def gather_order(chi_c: int, world: int):
    """For each rank, (lo, hi, padded length in slices) of its part of the gathered buffer."""
    per = max(hi - lo for lo, hi in (slice_range(chi_c, r, world) for r in range(world)))
    return [(*slice_range(chi_c, r, world), per) for r in range(world)]


def step_sharded(ctx, axis: int, chi: int, group=None, dist=None):
    """One coarse-graining of `ctx` along `axis`, its c'-slices split over the group."""
    import torch

    if dist is None:
        import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    on_device = dist.get_backend(group) == "nccl"
    dev = torch.device("cuda", torch.cuda.current_device()) if on_device else torch.device("cpu")
    n_grams, chi_c, per_slice = _b.shard_sizes(ctx, axis, chi)

    grams = torch.zeros(n_grams, dtype=torch.float64, device=dev)
    _b.hotrg_shard_env(ctx, axis, chi, rank, world, out=grams)
    dist.all_reduce(grams, group=group)
    _b.hotrg_shard_isometries(ctx, axis, chi, grams)

    parts = gather_order(chi_c, world)
    lo, hi, pad = parts[rank]
    mine = torch.zeros(pad * per_slice, dtype=torch.float64, device=dev)
    if hi > lo:
        _b.hotrg_shard_contract(ctx, axis, chi, lo, hi, out=mine[: (hi - lo) * per_slice])
    gathered = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(gathered, mine, group=group)
    full = torch.cat([g[: (h - l) * per_slice] for g, (l, h, _) in zip(gathered, parts)])
    _b.hotrg_shard_finish(ctx, axis, chi, full)
