"""The benchmark's multi-rank path (one independent grid per rank, weak
scaling): its only collective is the max over ranks of the timed interval.
Exercised with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_info() == (rank, world, rank)
        # rank r was slower or faster; every rank processed 1e6 updates
        elapsed = [250.0, 400.0][rank]
        mlups, t_max = bench.aggregate_ranks(elapsed, 1e6, world)
        dist.barrier()
        results[rank] = (mlups, t_max)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        results = m.dict()
        mp.spawn(_rank, args=(2, port, results), nprocs=2, join=True)
        got = dict(results)
    # both ranks agree: 2 ranks x 1e6 updates in the slower 0.4 s
    for r in (0, 1):
        mlups, t_max = got[r]
        assert t_max == 400.0
        assert abs(mlups - 2e6 / 0.4 / 1e6) < 1e-9


def test_single_rank_needs_no_collective():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    mlups, t_max = bench.aggregate_ranks(100.0, 5e6, 1)
    assert t_max == 100.0 and abs(mlups - 50.0) < 1e-12
