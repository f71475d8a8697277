"""The benchmark's multi-rank path on the CPU: two gloo ranks (replicas, one
per GPU on a real run) agree on the job's time as the slowest rank's, and the
job's throughput counts every rank's units over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(100.0 + 25.0 * rank, tdist, "cpu")
        units_per_rank = 1000.0
        out[rank] = (ms, units_per_rank * world / (ms / 1e3))
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1], "every rank reports the same job time and throughput"
    ms, value = res[0]
    assert ms == 125.0
    assert value == pytest.approx(2 * 1000.0 / 0.125)


def test_one_rank_needs_no_collective():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.5, None, "cpu") == 42.5
