"""Multi-rank host logic on CPU with torch.distributed gloo, world size 2."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2503_01471_gb300 import scenes as S
from paper_2503_01471_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, envs_per_rank, out):
    import torch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ids = list(shard.weak_shard(envs_per_rank, rank, world))
        batch, spec, poses = S.obstacle_rooms(envs_per_rank, steps=2, width=8, height=8, envs=ids)
        # what each rank would report: its rays and its (fake) step time; max over ranks
        t = torch.tensor([1.0 + rank], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        counts = torch.tensor([int(batch.env_tri_counts().sum())], dtype=torch.int64)
        gathered = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(gathered, counts)
        out[rank] = {"ids": ids, "max_t": float(t.item()), "tris": [int(g.item()) for g in gathered],
                     "first_pose": poses[0, 0].tolist()}
    finally:
        dist.destroy_process_group()


def test_weak_sharding_two_ranks():
    world, per = 2, 3
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, per, out), nprocs=world, join=True)
    ids0, ids1 = out[0]["ids"], out[1]["ids"]
    assert ids0 == [0, 1, 2] and ids1 == [3, 4, 5]
    assert out[0]["max_t"] == out[1]["max_t"] == 2.0
    # each rank's shard is exactly the single-process scene of those envs
    full, _, full_poses = S.obstacle_rooms(2 * per, steps=2, width=8, height=8)
    tri = full.env_tri_counts()
    assert out[0]["tris"] == [int(tri[:per].sum()), int(tri[per:].sum())]
    assert np.allclose(out[1]["first_pose"], full_poses[0, per])


def test_balanced_shards_cover_and_balance():
    rng = np.random.default_rng(0)
    tris = np.exp(rng.uniform(np.log(1e3), np.log(2e5), 8192)).astype(np.int64)
    rays = rng.choice([32400, 129600, 32768], 8192)
    costs = shard.env_cost(rays, tris)
    for world in (1, 2, 4, 8):
        sh = shard.balanced_shards(costs, world)
        flat = sorted(e for s in sh for e in s)
        assert flat == list(range(8192))
        assert shard.imbalance(costs, sh) < 1.001
    with pytest.raises(ValueError):
        shard.weak_shard(4, 2, 2)
