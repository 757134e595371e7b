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


def _costs(count, seed):
    from paper_2502_10685_gb300 import units, workloads as W
    items = W.uneven_batch(count, seed=seed)
    return [units.unit_cost(it.circuit.n, it.circuit.m,
                            it.circuit.n if it.kind == "generators" else 1) for it in items]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_lpt_partition_covers_every_item_once_and_balances(world):
    from paper_2502_10685_gb300 import units
    costs = _costs(600, seed=1003)
    parts = units.lpt_partition(costs, world)
    assert sorted(i for p in parts for i in p) == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    # the list-scheduling bound of LPT: no rank above the mean plus one item
    assert max(loads) <= sum(costs) / world + max(costs)
    assert parts == units.lpt_partition(costs, world)          # deterministic


def test_lpt_partition_small_cases():
    from paper_2502_10685_gb300 import units
    assert units.lpt_partition([], 2) == [[], []]
    assert units.lpt_partition([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    # LPT on {7, 6, 5, 4, 3, 3} over 2 ranks: 7+4+3 = 14 and 6+5+3 = 14
    parts = units.lpt_partition([7, 6, 5, 4, 3, 3], 2)
    assert sorted(sum([7, 6, 5, 4, 3, 3][i] for i in p) for p in parts) == [14, 14]
    with pytest.raises(ValueError):
        units.lpt_partition([1], 0)


def test_route_in_arrival_order():
    from paper_2502_10685_gb300 import units
    # least assigned work first, ties to the lower rank
    assert units.route_in_arrival_order([4, 1, 1, 1, 2], 2) == [0, 1, 1, 1, 1]
    assert units.route_in_arrival_order([1, 1, 1], 1) == [0, 0, 0]


def _gather_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2502_10685_gb300 import units
    costs = _costs(200, seed=7)
    mine = units.lpt_partition(costs, world)[rank]
    # each rank "runs" its units: the result of item i is a value only i gives
    results = [{"item": i, "value": i * 0.5} for i in mine]
    got = units.gather_to_root(mine, results, len(costs), dist)
    q.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gather_to_root_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(out[r] is None for r in range(1, world))
    full = out[0]
    assert [x["item"] for x in full] == list(range(len(full)))
    assert all(x["value"] == x["item"] * 0.5 for x in full)


def test_gather_to_root_rejects_duplicates_and_gaps():
    from paper_2502_10685_gb300 import units
    assert units.gather_to_root([1, 0], ["b", "a"], 2) == ["a", "b"]
    with pytest.raises(ValueError):
        units.gather_to_root([0, 0], ["a", "b"], 2)
    with pytest.raises(ValueError):
        units.gather_to_root([0], ["a"], 2)
