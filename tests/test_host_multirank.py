"""The N-GPU bench path on the host: with one process per GPU, each rank
searches its own disjoint slice of queries (weak scaling, no data-path
collective) and the job's time is the slowest rank's.  Run here as two gloo
ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, nq):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.shard_queries(rank, world, nq=nq)
        assert mine.shape == (nq, bench.DIM)
        shards = [None] * world
        dist.all_gather_object(shards, mine)
        full = bench.make_workload(n=1, nq=nq * world)[1]
        assert np.array_equal(np.concatenate(shards), full)  # disjoint slices covering one draw
        # the slowest rank's time sets the job's throughput
        local_ms = 10.0 + 5.0 * rank
        worst = bench.max_over_ranks(local_ms, world)
        assert worst == 10.0 + 5.0 * (world - 1)
        assert bench.job_qps(world, nq, 3, worst) == world * nq * 3 / (worst / 1e3)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_shard_queries_and_take_the_slowest_time(world):
    mp.spawn(_rank, args=(world, _free_port(), 64), nprocs=world, join=True)


def test_one_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_qps(1, 10000, 200, 320.0) == 10000 * 200 / 0.32
