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


def _shard_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import ffe_workloads as W
    from paper_2404_01531_gb300.partition import instance_work, instances_of
    cfgs = W.pulsars()
    mine = instances_of(cfgs, world, rank)
    lists = [None] * world
    dist.all_gather_object(lists, mine)
    work = torch.tensor([float(sum(instance_work(cfgs[i]) for i in mine))], dtype=torch.float64)
    tot = work.clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    out[rank] = (lists, work.item(), tot.item())
    dist.destroy_process_group()


def test_batch_instances_shard_over_two_gloo_ranks():
    """The 32-shell batch split by whole instances over two ranks: every rank
    derives the same assignment on its own, the shares are disjoint and cover
    every instance once, the ranks' work sums to the whole, and the larger
    share exceeds half the work by at most one instance's work (greedy
    longest-processing-time)."""
    import ffe_workloads as W
    from paper_2404_01531_gb300.partition import instance_work
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_shard_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    cfgs = W.pulsars()
    lists0 = out[0][0]
    assert out[1][0] == lists0
    flat = sorted(i for lst in lists0 for i in lst)
    assert flat == list(range(len(cfgs)))
    total = sum(instance_work(c) for c in cfgs)
    assert out[0][2] == out[1][2] == total
    big = max(instance_work(c) for c in cfgs)
    assert max(out[0][1], out[1][1]) <= total / 2 + big
    assert out[0][1] + out[1][1] == total


def test_instance_assignment_single_rank_and_errors():
    import ffe_workloads as W
    from paper_2404_01531_gb300.partition import assign_instances, instances_of
    cfgs = W.pulsars(n_inst=5)
    assert assign_instances(cfgs, 1) == [0] * 5
    assert instances_of(cfgs, 1, 0) == list(range(5))
    assert sorted(instances_of(cfgs, 8, 0) + [i for r in range(1, 8) for i in instances_of(cfgs, 8, r)]) == list(range(5))
    with pytest.raises(ValueError):
        assign_instances(cfgs, 0)
