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


def _step_shard_worker(rank, world, port, out):
    """Each rank steps its shard of small lattice scenes with the FP64 oracle
    (the stand-in for its GPU on this CPU test) and rank 0 gathers the
    accepted positions and velocities of every scene."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["OMP_NUM_THREADS"] = "1"
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import relcp_oracle as O

    scs = shard_test_scenes()
    a, b = shard_scenes([sc.n for sc in scs], world)[rank]
    flat = []
    for sc in scs[a:b]:
        flat.append(step_scene(O, sc))
    mine = torch.tensor(np.concatenate(flat) if flat else np.zeros(0), dtype=torch.float64)
    sizes = torch.tensor([mine.numel()], dtype=torch.int64)
    all_sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(all_sizes, sizes)
    cap = int(max(s.item() for s in all_sizes))
    pad = torch.zeros(cap, dtype=torch.float64)
    pad[:mine.numel()] = mine
    got = [torch.zeros(cap, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(got, pad)
    if rank == 0:
        out.put(np.concatenate([g[:int(s.item())].numpy() for g, s in zip(got, all_sizes)]))
    dist.barrier()
    dist.destroy_process_group()


def shard_test_scenes():
    return scenes.batched_scenes(n_scenes=12, seed0=700, nmax=48)


def step_scene(O, sc, steps=3):
    amin = float(sc.axes.min())
    cfg = O.Config(dynamics=O.INERTIAL, dt=sc.dt, eps_ncp=1e-3 * amin, box=tuple(sc.box), skin=0.1 * amin)
    x, q, v = sc.x, sc.q, sc.vel
    for _ in range(steps):
        r = O.step(cfg, x, q, sc.axes, v)
        x, q, v = r.x, r.q, r.vel
    return np.concatenate([x.ravel(), q.ravel(), v.ravel()])


def test_sharded_steps_merge_to_the_single_process_result(orc):
    """Two gloo ranks each step their contiguous shard of 12 independent
    scenes (no collective on the data path); the gathered result equals
    stepping every scene in one process, bit for bit."""
    world, port = 2, 29563
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_step_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    single = np.concatenate([step_scene(orc, sc) for sc in shard_test_scenes()])
    assert merged.shape == single.shape and np.array_equal(merged, single)
