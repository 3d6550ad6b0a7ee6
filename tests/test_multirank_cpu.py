"""The bench's multi-rank path on CPU: two gloo ranks, each timing its own replica, aggregate as
the slowest rank's time and the sum of the devices (weak scaling, no data-path collective)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        local_ms = [3.0, 5.0][rank]
        ms = bench.reduce_max(local_ms)
        out[rank] = (ms, bench.aggregate_value(world, 1000, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ms, v = res[rank]
        assert ms == 5.0
        assert v == pytest.approx(2 * 1000 / 5e-3)


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(2.5) == 2.5
    assert bench.aggregate_value(1, 393216, 0.25) == pytest.approx(393216 / 0.25e-3)
