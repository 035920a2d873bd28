"""Analyses the paper runs on batches of grown robots (Sec. 6.3, 6.4).

* Robustness (Sec. 6.3): the share of perturbed robots whose tip ends in the
  goal region, per uncertainty level.
* Funnelling (Sec. 6.4): how strongly contact concentrates the end points of
  trajectories that start from nearby conditions, measured by the k-nearest-
  neighbour density concentration ratio: for end point i, r_k(i) is the mean
  distance to its k nearest neighbours and p_i = k / (pi r_k(i)^2) its local
  density; the ratio is the mean density of the densest tenth of the points
  (p_i at or above the 90th percentile) over the mean density of all.

These run on the host on the results a batch returns (tips of a few thousand
robots); the simulation itself runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np


def success_rate(tips, goals, radius: float) -> float:
    """Share of robots whose tip lies within `radius` of its goal."""
    tips = np.asarray(tips, np.float64).reshape(-1, 2)
    goals = np.asarray(goals, np.float64).reshape(-1, 2)
    return float(np.mean(np.hypot(*(tips - goals).T) <= radius))


def knn_densities(points, k: int) -> np.ndarray:
    """p_i = k / (pi r_k(i)^2), r_k(i) the mean distance from point i to its
    k nearest other points."""
    p = np.asarray(points, np.float64).reshape(-1, 2)
    if len(p) <= k:
        raise ValueError("need more than k points")
    d = np.hypot(p[:, None, 0] - p[None, :, 0], p[:, None, 1] - p[None, :, 1])
    np.fill_diagonal(d, np.inf)
    rk = np.mean(np.sort(d, axis=1)[:, :k], axis=1)
    return k / (np.pi * rk ** 2)


def density_concentration_ratio(points, k: int = 5) -> float:
    """Mean density of the points at or above the 90th percentile of p over
    the mean density (1 for evenly spread points, larger when end points
    bunch up)."""
    p = knn_densities(points, k)
    top = p[p >= np.percentile(p, 90)]
    return float(np.mean(top) / np.mean(p))
