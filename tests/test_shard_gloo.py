"""Multi-rank host logic on CPU: world_size 2 with the gloo backend."""
import os
import socket

import pytest

from paper_1607_06283_gb300 import shard


def test_assign_streams_balances_and_covers():
    costs = [5, 1, 1, 1, 4, 4, 2, 2, 9, 3]
    parts = shard.assign_streams(costs, 3)
    assert sorted(sum(parts, [])) == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)
    assert shard.assign_streams(costs, 3) == parts  # deterministic
    assert shard.assign_streams([], 2) == [[], []]
    with pytest.raises(ValueError):
        shard.assign_streams(costs, 0)


def test_stream_seeds_differ_per_rank():
    seeds = {shard.stream_seed(1002, r) for r in range(8)}
    assert len(seeds) == 8 and shard.stream_seed(1002, 0) == 1002


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank "solves" its own streams; timing reduces to max, work to sum
        costs = [16384 * 50 * 40, 43200 * 50 * 20, 89960 * 50 * 10, 16384 * 50 * 5]
        mine = shard.assign_streams(costs, world)[rank]
        work = sum(costs[i] for i in mine)
        ms = 10.0 + rank
        dist.barrier()
        t, w = shard.reduce_timing(ms, work, dist)
        q.put((rank, mine, t, w))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    costs = [16384 * 50 * 40, 43200 * 50 * 20, 89960 * 50 * 10, 16384 * 50 * 5]
    assert sorted(res[0][1] + res[1][1]) == [0, 1, 2, 3]
    assert not set(res[0][1]) & set(res[1][1])
    for _, _, t, w in res:
        assert t == 11.0
        assert w == float(sum(costs))


def _batch_worker(rank, world, port, q):
    import torch.distributed as dist
    from evsim.configs import batch_configs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfgs = batch_configs()
        mine = shard.batch_share(cfgs, world, rank)
        work = sum(cfgs[i].W * cfgs[i].H * cfgs[i].iters * cfgs[i].n_packets for i in mine)
        dist.barrier()
        t, w = shard.reduce_timing(5.0 + rank, work, dist)
        q.put((rank, mine, work, t, w))
    finally:
        dist.destroy_process_group()


def test_batched_streams_split_over_two_gloo_ranks():
    """The 256-stream batched workload split over two ranks: every stream on exactly one
    rank, the work balanced, the timing reduced to the maximum and the work summed."""
    import torch.multiprocessing as mp
    from evsim.configs import batch_configs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfgs = batch_configs()
    costs = [c.W * c.H * c.iters * c.n_packets for c in cfgs]
    assert sorted(res[0][1] + res[1][1]) == list(range(256))
    assert abs(res[0][2] - res[1][2]) <= max(costs)
    for _, _, _, t, w in res:
        assert t == 6.0
        assert w == float(sum(costs))
