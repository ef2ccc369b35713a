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


def _seed_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2306_16705_gb300.vmc import sample_seed

    # the sampler seeds this rank's replica uses in its first 50 VMC steps
    mine = torch.tensor([sample_seed(bench.replica_seed(rank), t) for t in range(50)], dtype=torch.int64)
    got = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(got, mine)
    out[rank] = [g.tolist() for g in got]
    dist.destroy_process_group()


def test_replica_seeds_differ():
    """Two gloo ranks exchange the sampler seeds of their first 50 steps: no
    seed is used by both ranks (so their Philox streams, and the samples
    drawn from them, differ; tests/test_gpu_vmc.py draws with both)."""
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_seed_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    a, b = out[0]
    assert out[1] == [a, b]
    assert len(set(a)) == 50 and len(set(b)) == 50 and not set(a) & set(b)
