"""The benchmark's N > 1 path on CPU: two gloo ranks (replicas) agree on the
slowest rank's time and report whole-job throughput over it."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], world, device="cpu")
        out[rank] = (ms, bench.aggregate_throughput(10, world, ms))
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks_max_and_aggregate():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    times = [120.0, 200.0]
    mp.start_processes(_rank, args=(world, _free_port(), times, out), nprocs=world, start_method="spawn")
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 200.0
    assert value == pytest.approx(10 * 2 / 0.2)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(5.0, 1) == 5.0
    assert bench.aggregate_throughput(64, 1, 1000.0) == 64.0
