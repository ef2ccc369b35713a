"""The multi-rank form of the benchmark (independent replicas, one per GPU):
two gloo ranks on CPU check the aggregation -- the job's step time is the
slowest rank's and its work the sum of every rank's -- and that each rank
draws its own samples (distinct sampler seeds)."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, nu = bench.aggregate_ranks(10.0 + 3.0 * rank, 1000 * (rank + 1), dist, "cpu")
    out[rank] = (ms, nu)
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        ms, nu = out[r]
        assert ms == 13.0  # max over ranks
        assert nu == 3000  # sum over ranks


def test_replica_seeds_differ():
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py")).read()
    assert "seed=1000 + rank" in src
