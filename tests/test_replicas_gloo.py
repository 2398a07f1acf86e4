"""The multi-GPU path is replicas only: every rank evaluates its own netlist
instance on its own GPU with no collective on the data path; the job's time is
the max over ranks and its throughput sums all ranks.  This checks that host
logic with two gloo ranks on the CPU (no GPU involved)."""
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        my_ms = [12.5, 40.0][rank]  # the slower rank decides the job's time
        t = bench.replica_max_ms(my_ms, world)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(1000, rank))
        dist.barrier()
        out[rank] = (t, bench.replica_value(480, 3, world, t), seeds)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_max_time_and_sum_throughput():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        t, value, seeds = res[rank]
        assert t == 40.0
        assert value == pytest.approx(480 * 3 * 2 / 0.040)
        assert len(set(seeds)) == world  # distinct inputs per replica


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_max_ms(7.0, 1) == 7.0
    assert bench.replica_value(100, 2, 1, 50.0) == pytest.approx(4000.0)
