"""Scene sharding across ranks (host logic; two gloo processes on the CPU)."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2506_14097_gb300 import scenes
from paper_2506_14097_gb300.sharding import shard_cost, shard_scenes


def sizes_of_workload(n_scenes=2048):
    return [sc.n for sc in scenes.batched_scenes(n_scenes=n_scenes)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_shards_cover_and_balance(world):
    sizes = sizes_of_workload()
    sh = shard_scenes(sizes, world)
    assert sh[0][0] == 0 and sh[-1][1] == len(sizes)
    assert all(a <= b for a, b in sh) and all(sh[r][1] == sh[r + 1][0] for r in range(world - 1))
    cost = shard_cost(sizes, sh)
    # contiguous cuts: every shard within one largest scene of the ideal share
    ideal = sum(cost) / world
    assert max(abs(c - ideal) for c in cost) <= max(np.asarray(sizes, float) ** 2 + 1)


def test_shards_edge_cases():
    assert shard_scenes([], 3) == [(0, 0), (0, 0), (0, 0)]
    assert shard_scenes([5], 2) in ([(0, 1), (1, 1)], [(0, 0), (0, 1)])
    with pytest.raises(ValueError):
        shard_scenes([1, 2], 0)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = sizes_of_workload(512)
    a, b = shard_scenes(sizes, world)[rank]
    # each rank reports its own range and body count; rank 0 checks the union
    mine = torch.tensor([a, b, sum(sizes[a:b])], dtype=torch.int64)
    got = [torch.zeros(3, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(got, mine)
    if rank == 0:
        out.put([g.tolist() for g in got])
    dist.barrier()
    dist.destroy_process_group()


def test_ranks_agree_on_disjoint_cover():
    world, port = 2, 29561
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    sizes = sizes_of_workload(512)
    assert res[0][0] == 0 and res[-1][1] == len(sizes) and res[0][1] == res[1][0]
    assert sum(r[2] for r in res) == sum(sizes)
