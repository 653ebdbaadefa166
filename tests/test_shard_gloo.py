"""Multi-rank host logic of a batched run, on CPU with the gloo backend
(world size 2): every rank computes the same partition of the systems on its
own, the shares are disjoint and cover every system, the load is balanced, and
the step time is the maximum over ranks.  No GPU and no data-path collective."""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, sizes, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1607_04808_gb300 import shard
    costs = shard.system_costs("stokeslet", sizes, None, 8)
    parts = shard.partition(costs, world)
    mine = parts[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, {"parts": parts, "mine": mine})
    # a per-rank "step time"; the reported time is the maximum over ranks
    t = torch.tensor([1.0 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        torch.save({"gathered": gathered, "tmax": float(t.item()), "costs": costs},
                   os.path.join(out_dir, "shard.pt"))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_world2_gloo(tmp_path):
    from paper_1607_04808_gb300 import _build
    _build.build()
    import workloads as W
    sizes = [int(n) for n in W.lognormal_sizes(64, 5)]
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), sizes, str(tmp_path)), nprocs=world, join=True)
    res = torch.load(os.path.join(tmp_path, "shard.pt"))
    g = res["gathered"]
    assert g[0]["parts"] == g[1]["parts"]  # identical partition on every rank, no exchange needed
    mine = [set(x["mine"]) for x in g]
    assert not (mine[0] & mine[1])
    assert mine[0] | mine[1] == set(range(64))
    costs = res["costs"]
    loads = [sum(costs[i] for i in m) for m in mine]
    assert max(loads) <= 1.05 * sum(loads) / world
    assert res["tmax"] == 2.0


def test_partition_properties():
    from paper_1607_04808_gb300 import shard
    costs = [5.0, 1.0, 1.0, 1.0, 1.0, 1.0]
    assert shard.partition(costs, 2) == [[0], [1, 2, 3, 4, 5]]
    assert shard.partition(costs, 1) == [list(range(6))]
    parts = shard.partition([1.0] * 10, 3)
    assert sorted(i for p in parts for i in p) == list(range(10))
    assert [len(p) for p in parts] == [4, 3, 3]
    with pytest.raises(ValueError):
        shard.partition(costs, 0)
