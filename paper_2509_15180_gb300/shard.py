"""Partition of one batch's robots over several GPUs (one rank each).

Robots are independent: no step of the growth exchanges data between them,
so a batch shards with no collective on the data path.  The shards balance
the work by the longest-processing-time-first rule (Graham 1969): robots in
decreasing order of their cost estimate, each to the shard with the least
cost so far.  The estimate is the kernel's own queue key, N^2 (K_s n_obs + 8)
(N links, n_obs obstacles, K_s discs per link): the links present summed
over a growth are N (N + 1) / 2, and every link of every evaluation tests
K_s discs against the robot's obstacles.  LPT's largest shard is at most
4/3 of the optimum, and at most the mean shard plus the largest robot.
"""
from __future__ import annotations

import heapq

import numpy as np


def robot_cost(scene: dict, discs_per_link: int = 2) -> np.ndarray:
    """Cost estimate per robot: N^2 (K_s n_obs + 8)."""
    n = np.asarray(scene["n_links"], np.float64)
    n_obs = np.diff(np.asarray(scene["obs_ptr"], np.int64)).astype(np.float64)
    return n * n * (discs_per_link * n_obs + 8.0)


def lpt_partition(cost, n_parts: int) -> list[np.ndarray]:
    """Robot indices of each of n_parts shards (each sorted), by the LPT
    rule; ties (equal cost, equal load) go to the lower index, so every rank
    computes the same partition."""
    cost = np.asarray(cost, np.float64)
    if n_parts < 1:
        raise ValueError("n_parts must be positive")
    order = np.lexsort((np.arange(cost.size), -cost))  # decreasing cost, then index
    heap = [(0.0, p) for p in range(n_parts)]
    parts = [[] for _ in range(n_parts)]
    for i in order:
        load, p = heapq.heappop(heap)
        parts[p].append(int(i))
        heapq.heappush(heap, (load + float(cost[i]), p))
    return [np.sort(np.asarray(x, np.int64)) for x in parts]
