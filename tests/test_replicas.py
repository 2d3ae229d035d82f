"""Replica timing across ranks (bench.py under torchrun: one process per GPU, each advancing its
own problems, no data exchange): the job's time is the slowest rank's and its work the sum of
every rank's.  Checked with two gloo ranks on the CPU."""
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
        units = 1000 * (rank + 1)          # uneven work per rank
        ms = 10.0 + 5.0 * rank             # rank 1 is the slowest
        value, ms_max = bench.job_throughput(units, ms, 3, dist, "cpu")
        out[rank] = (value, ms_max, bench.reduce_over_ranks(rank + 1, dist, "cpu", "sum"))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_total_work_over_slowest_time():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in range(world):
        value, ms_max, s = res[rank]
        assert ms_max == 15.0                            # the slowest rank's time
        assert value == pytest.approx(3000 * 3 / 15e-3)  # all units over that time
        assert s == 3.0


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.job_throughput(500, 20.0, 4, None, "cpu")
    assert ms == 20.0 and value == pytest.approx(500 * 4 / 20e-3)
