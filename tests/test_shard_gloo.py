"""Sharding of independent slabs across ranks, on CPU with the gloo backend.

The phase-separation batch (256 independent slabs) is the part of the path
that partitions: each rank advances its LPT share and only per-slab results
are gathered at the end.  These tests run the host logic with world_size 2
(and 3) gloo ranks on CPU: every slab is advanced by exactly one rank, the
gather puts results back in slab order, and the shares are balanced within
the LPT bound; the partition itself is checked against brute force on tiny
cases.
"""
import itertools
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import json

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2503_15187_gb300 import shard
    from paper_2503_15187_gb300 import workloads as W
    slabs = W.batch_slabs(nslab=256)
    mine = shard.my_share(slabs, rank, world)
    # host stand-in for a slab's result: its total mass per unit length
    local = {i: float(slabs[i]["n0"].mean()) for i in mine}
    gathered = shard.gather_by_slab(local, len(slabs))
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"mine": mine, "gathered": gathered}, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_batch_shards_over_gloo_ranks(tmp_path, world):
    import json

    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from paper_2503_15187_gb300 import shard
    from paper_2503_15187_gb300 import workloads as W
    mp.spawn(_worker, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    slabs = W.batch_slabs(nslab=256)
    owned = sorted(i for r in res for i in r["mine"])
    assert owned == list(range(256))                       # each slab exactly once
    expect = [float(s["n0"].mean()) for s in slabs]
    for r in res:
        assert r["gathered"] == expect                     # slab order on every rank
    costs = shard.slab_costs(slabs)
    loads = [sum(costs[i] for i in r["mine"]) for r in res]
    lower = max(sum(costs) / world, max(costs))
    # with 256 slabs LPT is close to perfect: within 5 % of a lower bound of the optimum
    assert max(loads) <= 1.05 * lower


def test_lpt_against_brute_force():
    rng = np.random.default_rng(1)
    for trial in range(40):
        n, world = int(rng.integers(1, 8)), int(rng.integers(1, 4))
        costs = list(rng.integers(1, 50, n))
        from paper_2503_15187_gb300.shard import lpt_partition
        parts = lpt_partition(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(n))
        got = max(sum(costs[i] for i in p) for p in parts)
        best = min(max(sum(c for c, a in zip(costs, assign) if a == r) for r in range(world))
                   for assign in itertools.product(range(world), repeat=n))
        assert got <= (4.0 / 3.0 - 1.0 / (3 * world)) * best + 1e-9   # Graham's LPT bound


def test_single_rank_gets_everything():
    from paper_2503_15187_gb300.shard import lpt_partition
    assert lpt_partition([3, 1, 2], 1) == [[0, 1, 2]]
    with pytest.raises(ValueError):
        lpt_partition([1], 0)
