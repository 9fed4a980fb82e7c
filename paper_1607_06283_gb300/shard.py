"""Stream sharding across ranks (one process per GPU).

Event streams are independent (each has its own sensor, time surface and image), so
N GPUs share a workload by splitting the set of streams; no collective touches the
data path.  Only the timing of a benchmark is reduced across ranks: the elapsed time
is the maximum over ranks and the work is the sum.
"""
from __future__ import annotations


def assign_streams(costs, world: int) -> list:
    """Split stream indices over `world` ranks so that the summed cost per rank is
    balanced (longest-processing-time-first; ties by index, deterministic).

    costs: per-stream work (e.g. pixels x iterations x packets).  Returns a list of
    `world` sorted index lists."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(o) for o in out]


def batch_share(cfgs, world: int, rank: int) -> list:
    """Indices of the batched streams rank `rank` of `world` solves: the streams are
    balanced by their work (pixels x iterations x packets) with assign_streams."""
    costs = [c.W * c.H * c.iters * c.n_packets for c in cfgs]
    return assign_streams(costs, world)[rank]


def stream_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s own stream in a weak-scaling run (rank 0 keeps the base)."""
    return base_seed + 7 * rank


def reduce_timing(elapsed_ms: float, work: float, dist=None, device=None):
    """(max elapsed over ranks, summed work over ranks); identity without a process
    group.  `dist` is torch.distributed (any backend), `device` the tensor device."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(elapsed_ms), float(work)
    import torch
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())
