"""The N>1 path of the benchmark (replicas only: every rank runs its own job,
throughput is summed over ranks, time is the maximum over ranks), exercised
with two gloo ranks on the CPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = 1.0 + rank  # rank 1 is slower
    work_local = 100.0 * (rank + 1)
    t_max, work = bench.aggregate_ranks(t_local, work_local)
    out[rank] = (t_max, work)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn",
                       join=True)
    for r in range(world):
        t_max, work = out[r]
        assert t_max == 2.0  # max over ranks
        assert work == 300.0  # sum over ranks


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate_ranks(3.5, 7.0) == (3.5, 7.0)
