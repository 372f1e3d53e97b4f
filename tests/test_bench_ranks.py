"""The bench's cross-rank timing under a multi-process launch (world size 2,
gloo on the CPU): every rank steps its own replica, and the whole job is timed
as its slowest rank, so the reported time is the maximum over the ranks and
the throughput is all ranks' work over that time."""
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 345.5][rank]
        total = bench.max_over_ranks(local_ms, world, "cpu")
        out[rank] = total
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    if not dist.is_gloo_available():
        pytest.skip("gloo backend not built")
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res == {0: 345.5, 1: 345.5}


def test_max_over_ranks_single_process_is_the_value():
    import bench

    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
