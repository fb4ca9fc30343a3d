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


def _rank_data(rank):
    import numpy as np
    g = np.random.Generator(np.random.PCG64(900 + rank))
    R, n = 50, 40
    spins = np.where(g.random((R, n)) < 0.5, -1, 1).astype(np.int8)
    cuts = g.integers(300, 340, size=R)
    energies = -2 * cuts + g.integers(-3, 4, size=R)
    return cuts, energies, spins


def _gather_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2305_07187_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cuts, energies, spins = _rank_data(rank)
    ttt = 0.004 if rank == 1 else None          # only rank 1 reached the target
    res = replicas.gather_best(cuts, energies, spins, dist, ttt_s=ttt)
    best = res["best"]
    out[rank] = (best["cut"], best["energy"], best["rank"], best["replica"], best["spins"].tolist(),
                 res["hist"], res["replicas"], res["ttt_s"])
    dist.destroy_process_group()


def test_two_cpu_ranks_gather_best_replica_histogram_and_ttt():
    """End-of-run gather over ranks: every rank receives the best replica of
    the whole job (largest cut, ties to the lower energy, then the lower rank
    and replica), its spins, the summed cut histogram and the earliest
    time-to-target of any rank; checked against a direct search over both
    ranks' data."""
    import numpy as np
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_gather_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    cands = []
    hist = {}
    for rank in range(world):
        cuts, energies, spins = _rank_data(rank)
        for r in range(cuts.size):
            cands.append((-int(cuts[r]), int(energies[r]), rank, r))
            hist[int(cuts[r])] = hist.get(int(cuts[r]), 0) + 1
    ncut, e, rank_b, r_b = min(cands)
    spins_b = _rank_data(rank_b)[2][r_b].tolist()
    for rank in range(world):
        cut, energy, brank, brep, bspins, h, nrep, ttt = out[rank]
        assert (cut, energy, brank, brep) == (-ncut, e, rank_b, r_b)
        assert bspins == spins_b
        assert h == dict(sorted(hist.items())) and nrep == 100
        assert ttt == 0.004


def test_gather_on_one_rank_without_process_group():
    import numpy as np
    from paper_2305_07187_gb300 import replicas
    cuts = np.array([5, 9, 9, 2])
    energies = np.array([-1, -7, -8, 0])
    spins = np.arange(8, dtype=np.int8).reshape(4, 2)
    res = replicas.gather_best(cuts, energies, spins)
    assert res["best"]["cut"] == 9 and res["best"]["replica"] == 2 and res["best"]["energy"] == -8
    assert res["hist"] == {2: 1, 5: 1, 9: 2} and res["ttt_s"] is None
