"""Multi-rank host logic of bench.py on CPU ranks (gloo, world size 2): the
path shards replicas across ranks with no data-path collective; only the
timing scalar is reduced (maximum over ranks)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 + 5.0 * rank            # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms_local, dist)
    seeds = (bench.replica_seed0(rank), bench.replica_seed0(rank) + bench.REPLICAS)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    value = bench.whole_job_value(bench.REPLICAS * bench.N_SPINS * bench.T_STEPS, world, ms_max)
    out[rank] = (ms_max, gathered, value)
    dist.destroy_process_group()


def test_two_cpu_ranks_shard_replicas_and_take_the_max_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    import bench
    units = bench.REPLICAS * bench.N_SPINS * bench.T_STEPS
    for rank in range(world):
        ms_max, gathered, value = out[rank]
        assert ms_max == 15.0
        (a0, a1), (b0, b1) = gathered
        assert a1 <= b0 or b1 <= a0           # disjoint replica seed ranges
        assert value == pytest.approx(world * units / 15e-3)


def test_single_rank_without_process_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_value(100, 1, 1.0) == pytest.approx(1e5)
