"""The benchmark's N > 1 host logic (replicas, one per rank) on CPU: two gloo
ranks with different timed-region lengths agree on the slowest rank's time,
and the whole-job rate counts every rank's units over that time."""

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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank  # rank 1 is the slower replica
        t_max = bench.max_over_ranks(ms, dist)
        rate = bench.whole_job_rate(1000.0, world, t_max * 1e-3)
        out[rank] = (t_max, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_units():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    t_max, rate = res[0]
    assert t_max == 150.0
    assert rate == pytest.approx(2 * 1000.0 / 0.150)


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
