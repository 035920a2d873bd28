"""Pins of the planner oracle (oracle/sst.py) against hand-worked cases and
invariants of the pruning and selection rules of Sec. 5.2 (Algorithm 2)."""
import math

import numpy as np

from oracle import sst


def test_distance_closed_forms():
    assert sst.se2_dist2((0, 0, 0), (3, 4, 0), 10.0) == 25.0
    assert sst.se2_dist2((1, 2, 0.5), (1, 2, 0.5), 7.0) == 0.0
    # heading only: (rho * dphi)^2
    assert sst.se2_dist2((0, 0, 0.25), (0, 0, -0.25), 4.0) == 4.0  # (4 x 0.5)^2
    # wrap: headings 3 and -3 are 2 pi - 6 apart, not 6
    d2 = sst.se2_dist2((0, 0, 3.0), (0, 0, -3.0), 1.0)
    assert abs(math.sqrt(d2) - (2 * math.pi - 6.0)) < 1e-6
    d2 = sst.se2_dist2((0, 0, -3.0), (0, 0, 3.0), 1.0)
    assert abs(math.sqrt(d2) - (2 * math.pi - 6.0)) < 1e-6


def test_distance_is_a_metric_on_samples():
    rng = np.random.default_rng(0)
    P = np.stack([rng.uniform(-50, 50, 60), rng.uniform(-50, 50, 60), rng.uniform(-math.pi, math.pi, 60)], 1)
    P = P.astype(np.float32)
    for _ in range(300):
        a, b, c = P[rng.integers(0, 60, 3)]
        dab = math.sqrt(sst.se2_dist2(a, b, 30.0))
        assert dab == math.sqrt(sst.se2_dist2(b, a, 30.0))
        assert dab <= math.sqrt(sst.se2_dist2(a, c, 30.0)) + math.sqrt(sst.se2_dist2(c, b, 30.0)) + 1e-3


def _poses(*xy):
    return np.array([(x, y, 0.0) for x, y in xy], np.float32)


EMPTY_POSE = np.zeros((0, 3), np.float32)
EMPTY = np.zeros(0)


def test_prune_chain():
    """x (cost 3) overlaps y (cost 2), y overlaps z (cost 1), x and z are
    apart: y removes x and z removes y, so only z stays -- the region of x
    is left empty, as the rule 'keep the lowest of the overlapping' says."""
    new = _poses((0, 0), (8, 0), (16, 0))
    keep, _ = sst.prune(EMPTY_POSE, EMPTY, EMPTY, new, np.array([3.0, 2.0, 1.0]), 10.0, 1.0)
    assert keep.tolist() == [0, 0, 1]
    # reversed costs: x is the lowest and stays; y is removed by x, and z by
    # y, although y does not stay
    keep, _ = sst.prune(EMPTY_POSE, EMPTY, EMPTY, new, np.array([1.0, 2.0, 3.0]), 10.0, 1.0)
    assert keep.tolist() == [1, 0, 0]


def test_prune_against_the_tree():
    old = _poses((0, 0), (100, 0), (200, 0))
    old_cost = np.array([5.0, 1.0, 2.0])
    active = np.array([1, 1, 0], np.uint8)
    new = _poses((3, 4), (100, 6), (200, 1), (50, 0))
    new_cost = np.array([4.0, 1.5, 9.0, 7.0])
    keep, deact = sst.prune(old, old_cost, active, new, new_cost, 10.0, 1.0)
    # new 0 (cost 4, 5 from old 0 of cost 5): kept, old 0 deactivated
    # new 1 (cost 1.5, 6 from old 1 of cost 1): pruned
    # new 2 overlaps only the inactive old 2: kept
    # new 3 overlaps nothing: kept
    assert keep.tolist() == [1, 0, 1, 1]
    assert deact.tolist() == [1, 0, 0]


def test_prune_ties_go_to_the_tree_then_the_lower_index():
    old = _poses((0, 0))
    new = _poses((1, 0), (30, 0), (31, 0))
    keep, deact = sst.prune(old, np.array([2.0]), np.array([1], np.uint8), new, np.array([2.0, 3.0, 3.0]), 5.0, 1.0)
    assert keep.tolist() == [0, 1, 0] and deact.tolist() == [0]


def test_prune_boundary_is_strict():
    # exactly r apart: not overlapping
    new = _poses((0, 0), (3, 4))
    keep, _ = sst.prune(EMPTY_POSE, EMPTY, EMPTY, new, np.array([1.0, 2.0]), 5.0, 1.0)
    assert keep.tolist() == [1, 1]
    keep, _ = sst.prune(EMPTY_POSE, EMPTY, EMPTY, new, np.array([1.0, 2.0]), 5.0001, 1.0)
    assert keep.tolist() == [1, 0]


def test_prune_radius_limits():
    rng = np.random.default_rng(1)
    old = np.stack([rng.uniform(0, 100, 30), rng.uniform(0, 100, 30), rng.uniform(-3, 3, 30)], 1).astype(np.float32)
    new = np.stack([rng.uniform(0, 100, 40), rng.uniform(0, 100, 40), rng.uniform(-3, 3, 40)], 1).astype(np.float32)
    oc, nc = rng.uniform(0, 10, 30), rng.uniform(0, 10, 40)
    act = np.ones(30, np.uint8)
    # r = 0: nothing overlaps
    keep, deact = sst.prune(old, oc, act, new, nc, 0.0, 5.0)
    assert keep.all() and not deact.any()
    # r beyond every distance: the single lowest key among all states survives
    keep, deact = sst.prune(old, oc, act, new, nc, 1e4, 5.0)
    if nc.min() < oc.min():
        assert keep.sum() == 1 and keep[np.argmin(nc)] == 1 and deact.all()
    else:
        assert keep.sum() == 0 and not deact.any()


def test_prune_non_finite_cost_is_never_kept():
    new = _poses((0, 0), (50, 0))
    keep, _ = sst.prune(EMPTY_POSE, EMPTY, EMPTY, new, np.array([np.nan, np.inf]), 1.0, 1.0)
    assert keep.tolist() == [0, 0]


def test_prune_separation_invariant():
    """After pruning, the active tree nodes and the kept states are pairwise
    at least r apart, provided the active tree nodes were."""
    rng = np.random.default_rng(2)
    r, rho = 6.0, 8.0
    # a tree that is already sparse: greedy pick of separated points
    cand = np.stack([rng.uniform(0, 60, 400), rng.uniform(0, 60, 400), rng.uniform(-3, 3, 400)], 1).astype(np.float32)
    old = []
    for p in cand:
        if all(sst.se2_dist2(p, q, rho) >= np.float32(r * r) for q in old):
            old.append(p)
    old = np.array(old, np.float32)
    oc = rng.uniform(0, 10, len(old))
    act = np.ones(len(old), np.uint8)
    new = np.stack([rng.uniform(0, 60, 80), rng.uniform(0, 60, 80), rng.uniform(-3, 3, 80)], 1).astype(np.float32)
    nc = rng.uniform(0, 10, 80)
    keep, deact = sst.prune(old, oc, act, new, nc, r, rho)
    surv = [p for p, d in zip(old, deact) if not d] + [p for p, k in zip(new, keep) if k]
    for a in range(len(surv)):
        for b in range(a + 1, len(surv)):
            assert sst.se2_dist2(surv[a], surv[b], rho) >= np.float32(r * r)
    assert 0 < keep.sum() < 80


def test_prune_one_equals_prune():
    rng = np.random.default_rng(3)
    old = np.stack([rng.integers(0, 20, 50), rng.integers(0, 20, 50), rng.uniform(-3, 3, 50)], 1).astype(np.float32)
    new = np.stack([rng.integers(0, 20, 30), rng.integers(0, 20, 30), rng.uniform(-3, 3, 30)], 1).astype(np.float32)
    oc = rng.integers(0, 4, 50).astype(np.float64)   # many equal costs
    nc = rng.integers(0, 4, 30).astype(np.float64)
    act = (rng.random(50) < 0.7).astype(np.uint8)
    keep, _ = sst.prune(old, oc, act, new, nc, 3.0, 0.5)
    assert [sst.prune_one(j, old, oc, act, new, nc, 3.0, 0.5) for j in range(30)] == keep.tolist()


def test_select_best_near_and_nearest():
    pose = _poses((0, 0), (4, 0), (50, 0), (60, 0))
    cost = np.array([3.0, 1.0, 0.5, 0.2])
    active = np.array([1, 1, 1, 0], np.uint8)
    samples = _poses((1, 0), (58, 0), (500, 0), (2, 0))
    out = sst.select(pose, cost, active, samples, 5.0, 1.0)
    # sample 0: nodes 0 and 1 within 5, node 1 cheaper
    # sample 1: node 3 is inactive; node 2 is 8 away (beyond delta): nearest active = node 2
    # sample 2: nothing within delta: nearest active = node 2 (450 away)
    # sample 3: nodes 0 (2 away) and 1 (2 away) within delta: node 1 cheaper
    assert out.tolist() == [1, 2, 2, 1]
    # equal costs: lower index; equal distances with nothing in delta: lower index
    out = sst.select(pose, np.array([1.0, 1.0, 1.0, 1.0]), np.ones(4, np.uint8), _poses((2, 0), (27, 0)), 5.0, 1.0)
    assert out.tolist() == [0, 1]
    assert sst.select(pose, cost, np.zeros(4, np.uint8), samples, 5.0, 1.0).tolist() == [-1] * 4


def test_vectorised_forms_equal_the_plain_rules():
    rng = np.random.default_rng(4)
    for trial in range(3):
        n_old, n_new = 60, 40
        old = np.stack([rng.integers(0, 15, n_old), rng.integers(0, 15, n_old),
                        rng.choice([-3.0, -1.0, 0.0, 1.0, 3.0], n_old)], 1).astype(np.float32)
        new = np.stack([rng.integers(0, 15, n_new), rng.integers(0, 15, n_new),
                        rng.choice([-3.0, -1.0, 0.0, 1.0, 3.0], n_new)], 1).astype(np.float32)
        oc = rng.integers(0, 5, n_old).astype(np.float64)
        nc = rng.integers(0, 5, n_new).astype(np.float64)
        nc[rng.integers(0, n_new)] = np.nan
        act = (rng.random(n_old) < 0.6).astype(np.uint8)
        r = [2.0, 3.0, 5.0][trial]
        keep, deact = sst.prune(old, oc, act, new, nc, r, 1.5)
        assert [sst.deactivate_one(i, old, oc, act, new, nc, keep, r, 1.5) for i in range(n_old)] == deact.tolist()
        samples = np.stack([rng.integers(0, 15, 50), rng.integers(0, 15, 50), rng.uniform(-3, 3, 50)],
                           1).astype(np.float32)
        sel = sst.select(old, oc, act, samples, r, 1.5)
        assert [sst.select_one(q, old, oc, act, r, 1.5) for q in samples] == sel.tolist()
