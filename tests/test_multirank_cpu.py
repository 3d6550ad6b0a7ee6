"""The bench's multi-rank path on CPU (two gloo ranks, no GPU).

* Timing: every rank times its own share; the job's step time is the slowest rank's and its
  work the sum of the ranks' devices (weak scaling, no collective on the data path).
* Sharding of the batch of circuits (Sec. II parallelism over independent instances; each
  circuit's block of the block-diagonal system is independent): rank r owns circuits r, r + N, ...
  Each rank builds its own batched context from its share with the library's host-side calls;
  the shares partition the circuits, and every circuit's unknowns, nonzeros and devices in its
  rank's context equal those of the same circuit in the monolithic context, so the ranks' blocks
  reassemble the monolithic block-diagonal system.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)


def _timing_worker(rank, world, port, out):
    import torch.distributed as dist
    _init(rank, world, port)
    import bench
    try:
        local_ms = [3.0, 5.0][rank]
        local_dev = [1000, 1500][rank]
        ms = bench.reduce_max(local_ms)
        n_all = bench.sum_over_ranks(local_dev)
        out[rank] = (ms, n_all, bench.aggregate_value(n_all, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_timing_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ms, n_all, v = res[rank]
        assert ms == 5.0 and n_all == 2500
        assert v == pytest.approx(2500 / 5e-3)


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(2.5) == 2.5
    assert bench.sum_over_ranks(393216) == 393216
    assert bench.aggregate_value(393216, 0.25) == pytest.approx(393216 / 0.25e-3)


def _per_circuit_sizes(eec, nets):
    """(unknowns, nonzeros, devices) of every circuit of a batched context, from the library's
    host-side calls (the device upload is allowed to fail without a GPU)."""
    import netgen
    merged = netgen.concat(nets)
    ctx = eec.eec_create()
    try:
        eec.eec_upload_batch(ctx, nets)
        eec.eec_set_model_cards(ctx, netgen.default_cards())
        eec.eec_color(ctx, n_dev=merged.n_dev)
        try:
            eec.eec_build_scatter(ctx)
        except eec.EECError as e:
            assert e.code == eec.EEC_ECUDA
        ro, no, do = eec.eec_get_batch_offsets(ctx, len(nets))
    finally:
        eec.eec_destroy(ctx)
    return np.stack([np.diff(ro), np.diff(no), np.diff(do)], axis=1).astype(np.int64)


def _shard_worker(rank, world, port, n_circ, out):
    import torch.distributed as dist
    _init(rank, world, port)
    import netgen
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as eec
    try:
        nets = netgen.batch_circuits(n_circ, seed=5)
        mine = netgen.shard(nets, world, rank)
        ids = list(range(n_circ))[rank::world]
        sizes = _per_circuit_sizes(eec, mine)
        gathered = [None] * world
        dist.all_gather_object(gathered, (ids, sizes.tolist()))
        out[rank] = gathered
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_circuit_shards_partition_the_batch_and_reassemble_its_blocks():
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import netgen
    from paper_2604_03079_gb300 import build
    build.build()
    import paper_2604_03079_gb300 as eec
    n_circ, world = 37, 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_shard_worker, args=(world, port, n_circ, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]                      # both ranks hold every rank's share
    ids = [i for r in range(world) for i in res[0][r][0]]
    assert sorted(ids) == list(range(n_circ))    # the shares partition the circuits
    mono = _per_circuit_sizes(eec, netgen.batch_circuits(n_circ, seed=5))
    re = np.zeros_like(mono)
    for r in range(world):
        rid, sz = res[0][r]
        re[rid] = np.asarray(sz)
    assert np.array_equal(re, mono)              # every circuit's block, unchanged
    assert re.sum(axis=0).tolist() == mono.sum(axis=0).tolist()
    # the shares are balanced to within a few circuits' worth of devices
    dev = [int(np.asarray(res[0][r][1])[:, 2].sum()) for r in range(world)]
    assert max(dev) - min(dev) <= 3 * int(mono[:, 2].max())


def test_shard_rejects_bad_ranks():
    sys.path.insert(0, ROOT)
    import netgen
    with pytest.raises(ValueError):
        netgen.shard(list(range(5)), 2, 2)
    assert netgen.shard(list(range(5)), 2, 1) == [1, 3]
