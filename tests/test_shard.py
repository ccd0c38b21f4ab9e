"""Specimen sharding for batches across ranks: a deterministic, disjoint and
balanced partition, and the max-over-ranks timing reduction, checked with two
gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest

from paper_2201_04565_gb300 import shard


def test_partition_is_a_disjoint_balanced_cover():
    rng = np.random.default_rng(0)
    costs = [int(c) for c in rng.integers(32, 512, size=512) ** 2]
    for world in (1, 2, 3, 4, 8):
        shares = shard.partition(costs, world)
        flat = sorted(q for sh in shares for q in sh)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[q] for q in sh) for sh in shares]
        # longest-processing-time bound: no share exceeds the mean by more than the largest item
        assert max(loads) - sum(loads) / world <= max(costs)
        assert shard.partition(costs, world) == shares  # deterministic


def test_partition_edge_cases():
    assert shard.partition([], 3) == [[], [], []]
    assert shard.partition([5], 2) == [[0], []]
    assert shard.partition([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        shard.partition([1], 0)


def _worker(rank, world, port, costs, out):
    import torch.distributed as td
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.my_share(costs, rank, world)
    t = shard.max_over_ranks(float(rank + 1) * 0.5)
    import torch
    sizes = [None] * world
    td.all_gather_object(sizes, mine)
    out.put((rank, t, sizes))
    td.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    costs = [int(c) for c in np.random.default_rng(1).integers(10, 1000, size=37)]
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, shares in res:
        assert t == 1.0  # max of 0.5 and 1.0
        assert shares == shard.partition(costs, 2)
    flat = sorted(x for sh in res[0][2] for x in sh)
    assert flat == list(range(len(costs)))
