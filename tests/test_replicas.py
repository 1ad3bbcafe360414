"""The multi-rank bench path on CPU: two gloo ranks, as `bench.py --gpus 2` runs them under
torchrun (replicas: each rank advances its own instances, and only the timing and the update
counts cross ranks)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(dist, 10.0 + 5.0 * rank)          # per-rank device time
        upd = bench.sum_over_ranks(dist, [1000.0 * (rank + 1), 7.0])  # per-rank counts
        out[rank] = (ms, upd, bench.shard(11, rank, world))
    finally:
        dist.destroy_process_group()


def test_shards_cover_every_instance_once():
    for count in (1, 7, 256):
        for world in (1, 2, 3, 8):
            got = sorted(i for r in range(world) for i in bench.shard(count, r, world))
            assert got == list(range(count))


def test_two_gloo_ranks_reduce_time_and_updates():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ms, upd, mine = res[rank]
        assert ms == 15.0                       # the slowest rank
        assert upd == [3000.0, 14.0]            # whole-job totals
        assert mine == list(range(rank, 11, 2))


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.sum_over_ranks(None, [1.0, 2.0]) == [1.0, 2.0]
