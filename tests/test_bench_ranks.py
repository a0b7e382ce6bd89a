"""Host logic of the replicated multi-GPU bench path, on CPU with gloo ranks:
the slowest rank's time decides, and throughput counts every rank's problem."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate_ranks(times[rank], 4, 1000, world, torch.device("cpu"))
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput():
    world = 2
    times = [40.0, 100.0]   # total ms over 4 steps on each rank
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        ms, value = out[r]
        assert ms == pytest.approx(25.0)               # slowest rank: 100 ms / 4 steps
        assert value == pytest.approx(2 * 1000 / 25e-3 / 1e6)
