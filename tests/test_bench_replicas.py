"""The multi-GPU path of the benchmark is replicas (the solve is not sharded):
each rank solves its own right-hand sides and the job's throughput is all
ranks' solves over the slowest rank's time.  Two gloo ranks on the CPU check
the host logic of that reduction and that the replicas draw distinct inputs."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        own_ms = [120.0, 250.0][rank]                     # rank 1 is the slow one
        max_ms, value = bench.reduce_over_ranks(own_ms, 15, world, torch.device("cpu"))
        seeds = [bench.replica_rhs_seed(rank, i) for i in range(8)]
        out[rank] = (max_ms, value, seeds)
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_to_the_slowest_rank_and_draw_distinct_inputs():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        max_ms, value, _ = res[rank]
        assert max_ms == 250.0                              # every rank sees the slowest time
        assert abs(value - 2 * 15 / 0.250) <= 1e-9          # all ranks' solves over it
    assert not set(res[0][2]) & set(res[1][2])              # replicas solve different right-hand sides


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    max_ms, value = bench.reduce_over_ranks(200.0, 15, 1, None)
    assert max_ms == 200.0 and abs(value - 75.0) <= 1e-12
