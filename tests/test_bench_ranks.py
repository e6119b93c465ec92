"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1).

Each rank owns independent work (its own lattice, or its share of the sweep
domains); the only cross-rank steps are the barrier and the reductions of the
timing and counts, which these tests exercise."""
import json
import os
import socket
import types

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(dist, 1.5 + rank, "cpu")
        sw = bench.combine_sweep(dist, 10.0 * (rank + 1), 3 + rank, 1, 2 * rank, 1000 + rank, "cpu")
        mine = bench.shard(list(range(256)), rank, world)
        # sweep-like domain sizes (sites vary up to 64x): dealt by cost
        sizes = [64 + (37 * k) % 449 for k in range(256)]
        by_cost = bench.shard(list(range(256)), rank, world, cost=lambda k: sizes[k] ** 2)
        dist.barrier()
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
            json.dump({"t": t, "sweep": sw, "mine": mine, "by_cost": by_cost,
                       "sites": sum(sizes[k] ** 2 for k in by_cost)}, fh)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    assert r[0]["t"] == r[1]["t"] == 2.5                          # max over ranks
    assert r[0]["sweep"] == r[1]["sweep"] == [20.0, 7, 2, 2, 2001]  # max wall, summed counts
    assert sorted(r[0]["mine"] + r[1]["mine"]) == list(range(256))  # disjoint shards cover all
    assert not set(r[0]["mine"]) & set(r[1]["mine"])
    # the cost deal covers everything once and balances the sites to within the
    # largest single domain
    assert sorted(r[0]["by_cost"] + r[1]["by_cost"]) == list(range(256))
    assert abs(r[0]["sites"] - r[1]["sites"]) <= 512 ** 2


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(None, 3.25, "cpu") == 3.25
    assert bench.combine_sweep(None, 1.0, 2, 3, 4, 5, "cpu") == (1.0, 2, 3, 4, 5)
    assert bench.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    assert bench.shard([1, 2, 3], 0, 1, cost=lambda v: v) == [1, 2, 3]


def test_cost_shard_balances_uneven_items():
    """Longest first to the least loaded rank: four ranks over sweep-like sizes
    carry within one item of each other, where round robin can be far apart."""
    sizes = [64 + (53 * k) % 449 for k in range(256)]
    cost = lambda k: sizes[k] ** 2
    loads = [sum(cost(k) for k in bench.shard(list(range(256)), r, 4, cost=cost)) for r in range(4)]
    assert max(loads) - min(loads) <= max(cost(k) for k in range(256))
    parts = [bench.shard(list(range(256)), r, 4, cost=cost) for r in range(4)]
    assert sorted(sum(parts, [])) == list(range(256))


def test_reference_arm_other_ranks_exit_without_work():
    args = types.SimpleNamespace(steps=1, warmup=1)
    assert bench.run_reference(args, world=2, rank=1) == 0
