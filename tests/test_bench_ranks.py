"""The N > 1 path of bench.py on the CPU: two gloo ranks combine their timings
as the slowest rank's time and the sum of their units (replicas, no exchange)."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.combine_ranks(10.0 * (rank + 1), 1000 * (rank + 1), dist, "cpu")
    dist.barrier()
    out[rank] = (ms, units)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_the_summed_units():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        assert out[r] == (20.0, 3000.0)


def test_single_process_needs_no_process_group():
    import bench
    assert bench.combine_ranks(5.0, 7, None, "cpu") == (5.0, 7.0)
