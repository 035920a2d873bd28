"""Oracle for the tree operations of the batched SST* planner (Sec. 5.2,
Algorithm 2): the SE(2) distance between tip poses, the pruning of
overlapping states, and best-near selection of the nodes to expand.

TEST INFRASTRUCTURE ONLY: the tests and ``bench.py``'s CPU baseline leg are
the only users; the product package never imports this module.  Written
plainly from the definitions below, one pair at a time, so that each rule
can be checked against the paper by eye.

Decisions (within the radius or not, which key is smaller) are integers
decided by floating point, so this side takes them in the precision the
kernel takes them in: the squared distance in IEEE float32, every product
and sum rounded on its own (no fused multiply-add), in the order written
in ``se2_dist2``.  Costs are compared exactly (float64).

Readings of the paper (Sec. 5.2):
* SE(2) metric: d^2 = dx^2 + dy^2 + (rho * dphi)^2, dphi the heading
  difference wrapped to [-pi, pi]; rho converts radians to the caller's
  length unit (the paper combines millimetres and radians with r_init = 60).
* Two states overlap when d < r (strictly).
* Pruning keeps a new state exactly when no overlapping state -- an active
  tree node or another new state -- has a smaller key; an active tree node is
  deactivated when a kept new state with a smaller key overlaps it.  Keys
  are (cost, id), tree nodes numbered before new states, so that ties go to
  the tree and then to the lower index.  A new state with a non-finite cost
  is never kept.
* Selection of a node to expand for a sample pose: the active node of
  smallest key among those within delta of the sample; if none is within
  delta, the nearest active node (smallest (d^2, index)); -1 when the tree
  has no active node.
"""
from __future__ import annotations

import math

import numpy as np

F32 = np.float32
PI_F32 = F32(math.pi)
TWO_PI_F32 = F32(2.0 * math.pi)


def se2_dist2(a, b, rho) -> np.float32:
    """Squared SE(2) distance between poses a = (x, y, phi) and b, headings
    in [-pi, pi]; float32, each operation rounded."""
    dx = F32(F32(a[0]) - F32(b[0]))
    dy = F32(F32(a[1]) - F32(b[1]))
    dp = F32(F32(a[2]) - F32(b[2]))
    if dp > PI_F32:
        dp = F32(dp - TWO_PI_F32)
    elif dp < -PI_F32:
        dp = F32(dp + TWO_PI_F32)
    rp = F32(F32(rho) * dp)
    return F32(F32(F32(dx * dx) + F32(dy * dy)) + F32(rp * rp))


def _within(a, b, rho, r) -> bool:
    r2 = F32(F32(r) * F32(r))
    return bool(se2_dist2(a, b, rho) < r2)


def prune(old_pose, old_cost, old_active, new_pose, new_cost, radius, rho):
    """Pruning of overlapping states.  Returns (keep[n_new], deactivate[n_old])
    as uint8 arrays.  One pair at a time: O((n_old + n_new) n_new)."""
    n_old, n_new = len(old_cost), len(new_cost)
    keep = np.zeros(n_new, np.uint8)
    deact = np.zeros(n_old, np.uint8)
    for j in range(n_new):
        cj = float(new_cost[j])
        if not math.isfinite(cj):
            continue
        kj = (cj, n_old + j)
        ok = True
        for i in range(n_old):
            if old_active[i] and (float(old_cost[i]), i) < kj and _within(new_pose[j], old_pose[i], rho, radius):
                ok = False
                break
        if ok:
            for k in range(n_new):
                ck = float(new_cost[k])
                if k != j and math.isfinite(ck) and (ck, n_old + k) < kj and \
                        _within(new_pose[j], new_pose[k], rho, radius):
                    ok = False
                    break
        keep[j] = ok
    for i in range(n_old):
        if not old_active[i]:
            continue
        ki = (float(old_cost[i]), i)
        for j in range(n_new):
            if keep[j] and (float(new_cost[j]), n_old + j) < ki and _within(old_pose[i], new_pose[j], rho, radius):
                deact[i] = 1
                break
    return keep, deact


def select(pose, cost, active, samples, delta, rho):
    """Best-near selection: for every sample pose, the index of the node to
    expand (-1 if no node is active)."""
    n = len(cost)
    out = np.full(len(samples), -1, np.int32)
    d2lim = F32(F32(delta) * F32(delta))
    for s, q in enumerate(samples):
        best = None
        near = None
        for i in range(n):
            if not active[i]:
                continue
            d2 = se2_dist2(q, pose[i], rho)
            if d2 < d2lim and (best is None or (float(cost[i]), i) < (float(cost[best]), best)):
                best = i
            if near is None or (d2, i) < near:
                near = (d2, i)
        if best is not None:
            out[s] = best
        elif near is not None:
            out[s] = near[1]
    return out


def prune_one(j, old_pose, old_cost, old_active, new_pose, new_cost, radius, rho):
    """keep[j] of ``prune`` for one new state, vectorised over the tree in
    float32 with the same rounding (for sampled checks at large sizes)."""
    n_old = len(old_cost)
    cj = float(new_cost[j])
    if not math.isfinite(cj):
        return 0
    r2 = F32(F32(radius) * F32(radius))
    d2 = _dist2_rows(new_pose[j], old_pose, rho)
    idx = np.arange(n_old)
    lower = (old_cost < cj) | ((old_cost == cj) & (idx < n_old + j))
    if np.any((old_active != 0) & lower & (d2 < r2)):
        return 0
    d2n = _dist2_rows(new_pose[j], new_pose, rho)
    k = np.arange(len(new_cost))
    fin = np.isfinite(new_cost)
    lowern = (new_cost < cj) | ((new_cost == cj) & (k < j))
    return int(not np.any(fin & lowern & (k != j) & (d2n < r2)))


def deactivate_one(i, old_pose, old_cost, old_active, new_pose, new_cost, keep, radius, rho):
    """deactivate[i] of ``prune`` for one tree node, given the keep flags of
    the new states, vectorised over them with the same float32 rounding."""
    if not old_active[i]:
        return 0
    ci = float(old_cost[i])
    r2 = F32(F32(radius) * F32(radius))
    d2 = _dist2_rows(old_pose[i], new_pose, rho)
    lower = new_cost < ci   # a new state's id is above every tree node's
    return int(np.any((np.asarray(keep) != 0) & lower & (d2 < r2)))


def select_one(q, pose, cost, active, delta, rho):
    """``select`` for one sample pose, vectorised over the nodes."""
    act = np.nonzero(np.asarray(active) != 0)[0]
    if act.size == 0:
        return -1
    d2 = _dist2_rows(q, np.asarray(pose)[act], rho)
    d2lim = F32(F32(delta) * F32(delta))
    inside = act[d2 < d2lim]
    if inside.size:
        c = np.asarray(cost)[inside]
        # smallest cost, then lowest index (inside is increasing)
        return int(inside[np.lexsort((inside, c))[0]])
    m = d2.min()
    return int(act[np.nonzero(d2 == m)[0][0]])


def _dist2_rows(a, P, rho):
    """se2_dist2(a, P[i]) for every row of P, the same float32 operations."""
    P = np.asarray(P, F32)
    dx = (F32(a[0]) - P[:, 0]).astype(F32)
    dy = (F32(a[1]) - P[:, 1]).astype(F32)
    dp = (F32(a[2]) - P[:, 2]).astype(F32)
    dp = np.where(dp > PI_F32, (dp - TWO_PI_F32).astype(F32), np.where(dp < -PI_F32, (dp + TWO_PI_F32).astype(F32), dp))
    rp = (F32(rho) * dp).astype(F32)
    return ((dx * dx).astype(F32) + (dy * dy).astype(F32)).astype(F32) + (rp * rp).astype(F32)
