"""Replica aggregation of bench.py on two gloo ranks (CPU): every rank gets the
slowest rank's time and the whole-job throughput counts both ranks' units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]
    total_ms, value = bench.combine_ranks(local_ms, 1000, world, dist, "cpu")
    q.put((rank, total_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, total_ms, value in out:
        assert total_ms == 250.0
        assert abs(value - 2 * 1000 / 0.25) < 1e-9


def test_combine_ranks_single():
    import bench
    total_ms, value = bench.combine_ranks(50.0, 10, 1)
    assert total_ms == 50.0 and abs(value - 200.0) < 1e-12


def test_batch_shards_cover_every_item_once():
    import bench
    items = list(range(4096 * 3))
    shards = [bench.shard(items, r, 3) for r in range(3)]
    assert sorted(x for sh in shards for x in sh) == items
    assert max(len(sh) for sh in shards) - min(len(sh) for sh in shards) <= 1
