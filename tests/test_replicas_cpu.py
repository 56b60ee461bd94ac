"""The multi-GPU form is replicas only (one independent copy of the workload per rank, no
collective on the data path); the bench combines the ranks' timings with a max. This runs that
host logic as two gloo ranks on the CPU."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_max, value = bench.combine_replicas(10.0 + 5.0 * rank, 4, 8 ** 3, dist, "cpu")
        out[rank] = (ms_max, value)
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_max_time_and_whole_job_throughput():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        got = dict(out)
    expect_ms = 15.0
    expect_value = world * 8 ** 3 * 4 / (expect_ms * 1e-3)
    for rank in range(world):
        ms_max, value = got[rank]
        assert ms_max == expect_ms
        assert abs(value - expect_value) < 1e-9 * expect_value


def test_single_process_is_its_own_maximum():
    sys.path.insert(0, ROOT)
    import bench

    ms_max, value = bench.combine_replicas(12.5, 10, 1000)
    assert ms_max == 12.5 and abs(value - 1000 * 10 / 12.5e-3) < 1e-6
