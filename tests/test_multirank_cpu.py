"""The multi-rank path of bench.py on CPU: world_size 2 over gloo, 127.0.0.1.

Each rank analyses its own HoMLN (replicas); the job's throughput is the units summed over the
ranks divided by the slowest rank's time. No data-path collective is involved."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, secs = bench.job_aggregate(100.0 * (rank + 1), 1.0 + rank, dist, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.replica_seed(2001, rank))
    out[rank] = (units, secs, seeds)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        units, secs, seeds = res[r]
        assert units == 300.0 and secs == 2.0  # summed work, slowest rank's time
        assert len(set(seeds)) == world  # every rank analyses its own HoMLN


def _shard_main(rank, world, port, out):
    """Each rank sums the BFS distances from its source batches (the oracle's BFS, batches of
    64 sources dealt round-robin as the library deals them); shard.reduce_partials sums them."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2207_11662_gb300 import shard, synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 700
    s, d = synth.chung_lu_edges(n, 2500, 91)
    rp, col = O.simple_csr(n, s, d)
    F = np.zeros(n, np.int64)
    R = np.zeros(n, np.int32)
    for b in range(rank, (n + 63) // 64, world):
        for src in range(64 * b, min(64 * (b + 1), n)):
            dist_s = O.bfs_dist(n, rp, col, src)
            reached = dist_s > 0
            F[reached] += dist_s[reached]
            R[reached] += 1
    Ft, Rt = torch.from_numpy(F), torch.from_numpy(R)
    shard.reduce_partials(Ft, Rt, dist)
    Fo, Ro = O.farness_reach(n, rp, col)
    out[rank] = bool(np.array_equal(Ft.numpy().astype(np.uint64), Fo) and np.array_equal(Rt.numpy(), Ro.astype(np.int32)))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_sources_reduce_to_the_full_analysis_gloo():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_shard_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert all(res[r] for r in range(world))
