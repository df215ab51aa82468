"""The multi-rank (replica) path of bench.py on CPU: two gloo ranks reduce
their timings the way the GPU ranks do -- the slowest rank's time and the sum
of all ranks' particle-steps."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, s = bench.reduce_times(dist, total_ms=10.0 + 5.0 * rank, steps_done=1000 * (rank + 1))
    out[rank] = (t, s)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_sum_steps():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        assert out[r] == (15.0, 3000.0)


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_times(None, 12.5, 77) == (12.5, 77)


def _shard_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    work = [float((7 * i) % 23 + 1) for i in range(50)]
    mine = bench.shard_by_work(work, world)[rank]
    # each rank's particle-steps summed and its time maxed, as run_batched does
    t, s = bench.reduce_times(dist, total_ms=1.0 + sum(work[i] for i in mine), steps_done=len(mine))
    out[rank] = (mine, t, s)
    dist.barrier()
    dist.destroy_process_group()


def test_batched_filters_shard_over_two_gloo_ranks():
    """The batched benchmark's sharding: every filter on exactly one rank, the
    ranks' work balanced to within the largest filter, the reduction giving
    the slowest rank's time and all filters."""
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_shard_worker, args=(world, port, out), nprocs=world, start_method="spawn",
                       join=True)
    work = [float((7 * i) % 23 + 1) for i in range(50)]
    shards = [out[r][0] for r in range(world)]
    assert sorted(i for s in shards for i in s) == list(range(50))
    loads = [sum(work[i] for i in s) for s in shards]
    assert max(loads) - min(loads) <= max(work)
    for r in range(world):
        assert out[r][1] == 1.0 + max(loads) and out[r][2] == 50
