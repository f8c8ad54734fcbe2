"""Environment sharding across GPUs (one process per GPU, no collective on the data path).

Environments are independent (Sec. III-D.1: each holds its own meshes and
BVH), so a multi-GPU run only partitions them. Weak scaling gives every rank
its own block of environments; for a fixed set of uneven environments the
greedy partition below balances an estimate of their traversal cost.
"""
from __future__ import annotations

import heapq
import math

import numpy as np


def weak_shard(envs_per_rank: int, rank: int, world: int) -> range:
    """Global environment indices of ``rank`` when every rank renders ``envs_per_rank`` envs."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return range(rank * envs_per_rank, (rank + 1) * envs_per_rank)


def env_cost(rays_per_env, tris_per_env) -> np.ndarray:
    """Traversal cost estimate of each env: rays x log2(triangles + 2)."""
    rays = np.broadcast_to(np.asarray(rays_per_env, np.float64), np.shape(tris_per_env))
    return rays * np.log2(np.asarray(tris_per_env, np.float64) + 2.0)


def balanced_shards(costs, world: int) -> list[list[int]]:
    """Greedy longest-processing-time partition of env indices into ``world`` shards.

    Envs are taken in decreasing cost and each goes to the currently lightest
    shard; ties go to the lower rank. Each shard lists its envs in ascending
    index order. The result covers every env exactly once.
    """
    costs = np.asarray(costs, np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0.0, r) for r in range(world)]
    shards: list[list[int]] = [[] for _ in range(world)]
    for e in sorted(range(costs.shape[0]), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        shards[r].append(e)
        heapq.heappush(heap, (load + float(costs[e]), r))
    return [sorted(s) for s in shards]


def imbalance(costs, shards) -> float:
    """max shard cost / mean shard cost (1.0 = perfect)."""
    costs = np.asarray(costs, np.float64)
    loads = [float(costs[s].sum()) for s in shards]
    mean = sum(loads) / len(loads)
    return max(loads) / mean if mean > 0 else 1.0
