"""The N > 1 bench path runs independent replicas (no data-path collective): the only
cross-rank steps are the barrier around the timed region and the max of the per-rank times.
Checked here with two gloo ranks on the CPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # rank r pretends its timed region took 10 + r milliseconds
        slowest = bench.max_over_ranks(world, 10.0 + rank)
        value = bench.aggregate(world, 1000.0, 5, slowest)
        out[rank] = (slowest, value)
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_sum_the_work():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        slowest, value = out[rank]
        assert slowest == 11.0
        assert abs(value - 2 * 1000.0 * 5 / 0.011) < 1e-6
