"""The multi-rank path of bench.py on CPU: two gloo ranks (one replica per
GPU on the real machine) reduce their timings to the whole-job figures:
max of the times, sum of the samples."""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, n = bench.reduce_over_ranks(100.0 + 10 * rank, 1000 * (rank + 1), torch.device("cpu"))
    out[rank] = (t, n)
    dist.destroy_process_group()


def test_two_rank_reduction():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        assert out[r] == (110.0, 3000.0)


def test_single_process_passthrough():
    import bench
    assert bench.reduce_over_ranks(12.5, 7, torch.device("cpu")) == (12.5, 7.0)
