"""Splitting a batch of instances across ranks (one process per GPU).

Instances are independent and every path's random numbers are keyed by its
(instance, path) numbers, so a batch can be cut into contiguous instance
ranges with no exchange during the walk.  Each rank walks its range under
the instances' global numbers (``instance_offset``) and the per-instance
results are concatenated afterwards; nothing else is communicated.
"""
from typing import Callable, Tuple


def shard_range(n_inst: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [begin, end) of instances for `rank` out of `world`; the
    first n_inst % world ranks take one extra instance."""
    if world < 1 or not (0 <= rank < world) or n_inst < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_inst, world)
    begin = rank * base + min(rank, extra)
    end = begin + base + (1 if rank < extra else 0)
    return begin, end


def gather_instances(local, n_inst: int, group=None):
    """Concatenate per-rank per-instance arrays (torch tensors, first axis =
    local instances) into the full [n_inst, ...] array on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    sizes = [shard_range(n_inst, r, world) for r in range(world)]
    width = max(e - b for b, e in sizes)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:e - b] for p, (b, e) in zip(parts, sizes)], dim=0)


def shard_batch(x, rank: int, world: int):
    """This rank's contiguous share of a batch of walk inputs (an
    ``inputs.WalkInputs``) and the global number of its first instance."""
    import numpy as np
    b, e = shard_range(x.n_inst, rank, world)
    if (b, e) == (0, x.n_inst):
        return x, b
    return x.subset(np.arange(b, e)), b


def walk_and_gather(walk_fn: Callable, x_local, begin: int, n_total: int, group=None,
                    gather: bool = True):
    """Walks one rank's share and gathers the per-instance results.

    ``walk_fn(x_local, begin)`` walks the share under the instances' global
    numbers (``instance_offset = begin``) and returns torch tensors R [n] and
    bins [n][nbins].  The two are packed as one [n][1 + nbins] table, so the
    exchange is a single all_gather; with ``gather`` every rank ends with
    the [n_total][1 + nbins] table of the whole batch, in instance order."""
    import torch
    import torch.distributed as dist
    R, bins = walk_fn(x_local, begin)
    local = torch.cat([R.reshape(-1, 1), bins.reshape(R.shape[0], -1)], dim=1)
    if not gather or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return local
    return gather_instances(local, n_total, group)


def max_over_ranks(seconds: float, group=None) -> float:
    """The job's time: the slowest rank's."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
