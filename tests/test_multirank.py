"""The multi-rank logic of bench.py on the CPU: two gloo ranks (spawned
processes, rendezvous on 127.0.0.1).  Each rank shards the batched fields
without any exchange, and the job's time is the slowest rank's.  No GPU and
no collective on the data path: each rank's work is independent (fields, or
a whole field per rank)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ls, out_dir):
    import json
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = bench.shard_fields(ls, rank, world)
        shards = [None] * world
        dist.all_gather_object(shards, mine)
        slowest = bench.max_over_ranks(10.0 * (rank + 1), world, dist)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"mine": mine, "shards": shards, "slowest": slowest}, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_field_sharding_and_slowest_rank(tmp_path, world):
    import json

    import numpy as np
    import torch.multiprocessing as mp

    ls = [int(x) for x in np.random.default_rng(4).choice([64, 128, 256, 512, 1024], size=96)]
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, ls, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    # every rank computed the same assignment on its own
    for r in range(world):
        assert res[r]["shards"] == res[0]["shards"]
        assert res[r]["mine"] == res[0]["shards"][r]
        assert res[r]["slowest"] == 10.0 * world
    shards = res[0]["shards"]
    flat = sorted(f for s in shards for f in s)
    assert flat == list(range(len(ls)))  # disjoint, complete
    # balanced: loads differ by at most the largest single field's cost
    cost = [l * l * np.log2(l) for l in ls]
    loads = [sum(cost[f] for f in s) for s in shards]
    assert max(loads) - min(loads) <= max(cost)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.shard_fields([64, 1024, 128], 0, 1) == [0, 1, 2]
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
