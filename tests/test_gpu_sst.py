"""GPU parity of the planner's tree operations (vine_sst_prune,
vine_sst_select) against the oracle (oracle/sst.py): bit-exact flags and
indices, on inputs full of ties (integer grid poses, headings on a few
values that wrap, integer costs), at sizes spanning several tiles, chunks
and ragged tails, and sampled at large sizes."""
import math

import numpy as np
import pytest

from oracle import sst

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402

HEADINGS = np.array([-math.pi, -3.0, -1.0, 0.0, 1.0, 3.0, math.pi], np.float32)


def _poses(rng, n, span):
    return np.stack([rng.integers(0, span, n), rng.integers(0, span, n), rng.choice(HEADINGS, n)],
                    1).astype(np.float32)


def _case(seed, n_old, n_new, span=40):
    rng = np.random.default_rng(seed)
    old, new = _poses(rng, n_old, span), _poses(rng, n_new, span)
    oc = rng.integers(0, 6, n_old).astype(np.float64)
    nc = rng.integers(0, 6, n_new).astype(np.float64)
    if n_new > 3:
        nc[rng.integers(0, n_new, 2)] = np.nan
    act = (rng.random(n_old) < 0.7).astype(np.uint8)
    return old, oc, act, new, nc


@pytest.mark.parametrize("n_old,n_new,r", [(0, 0, 3.0), (0, 1, 3.0), (1, 0, 3.0), (0, 300, 4.0), (257, 129, 3.0),
                                           (1000, 700, 5.0), (3000, 513, 2.0)])
def test_prune_matches_oracle(n_old, n_new, r):
    old, oc, act, new, nc = _case(n_old * 7 + n_new, n_old, n_new)
    keep, deact = vine.sst_prune(old, oc, act, new, nc, r, 1.5)
    if n_old * n_new + n_new * n_new <= 600000:
        ok, od = sst.prune(old, oc, act, new, nc, r, 1.5)
    else:
        ok = np.array([sst.prune_one(j, old, oc, act, new, nc, r, 1.5) for j in range(n_new)], np.uint8)
        od = np.array([sst.deactivate_one(i, old, oc, act, new, nc, ok, r, 1.5) for i in range(n_old)], np.uint8)
    assert np.array_equal(keep, ok)
    assert np.array_equal(deact, od)
    print("prune %d/%d: kept %d, deactivated %d" % (n_old, n_new, keep.sum(), deact.sum()))


@pytest.mark.parametrize("n_nodes,n_s,delta", [(0, 5, 3.0), (1, 1, 3.0), (300, 129, 4.0), (2049, 700, 2.5),
                                               (5000, 1, 6.0)])
def test_select_matches_oracle(n_nodes, n_s, delta):
    rng = np.random.default_rng(n_nodes + 13 * n_s)
    pose = _poses(rng, n_nodes, 40)
    cost = rng.integers(0, 6, n_nodes).astype(np.float64)
    act = (rng.random(n_nodes) < 0.7).astype(np.uint8)
    samples = np.stack([rng.uniform(-5, 45, n_s), rng.uniform(-5, 45, n_s), rng.uniform(-math.pi, math.pi, n_s)],
                       1).astype(np.float32)
    samples[: n_s // 3, :2] = np.round(samples[: n_s // 3, :2])  # samples on the grid: exact ties
    got = vine.sst_select(pose, cost, act, samples, delta, 1.5)
    want = np.array([sst.select_one(q, pose, cost, act, delta, 1.5) for q in samples], np.int32)
    assert np.array_equal(got, want)


def test_prune_select_large_sampled():
    """Tree of 400k nodes, 4096 new states and samples (the planner's batch
    of expansions); 256 of each output checked one by one."""
    rng = np.random.default_rng(99)
    n_old, n_new = 400_000, 4096
    old = np.stack([rng.uniform(0, 2000, n_old), rng.uniform(0, 2000, n_old),
                    rng.uniform(-math.pi, math.pi, n_old)], 1).astype(np.float32)
    new = np.stack([rng.uniform(0, 2000, n_new), rng.uniform(0, 2000, n_new),
                    rng.uniform(-math.pi, math.pi, n_new)], 1).astype(np.float32)
    oc = rng.uniform(0, 8, n_old)
    nc = rng.uniform(0, 8, n_new)
    act = (rng.random(n_old) < 0.5).astype(np.uint8)
    r, rho = 12.0, 20.0
    keep, deact = vine.sst_prune(old, oc, act, new, nc, r, rho)
    for j in rng.choice(n_new, 256, replace=False):
        assert keep[j] == sst.prune_one(j, old, oc, act, new, nc, r, rho), j
    # tree nodes near kept new states, where deactivation can happen, and random ones
    near = np.nonzero(deact)[0]
    pick = np.concatenate([near[: 128], rng.choice(n_old, 128, replace=False)])
    for i in pick:
        assert deact[i] == sst.deactivate_one(i, old, oc, act, new, nc, keep, r, rho), i
    samples = new.copy()
    got = vine.sst_select(old, oc, act, samples, r, rho)
    for s in rng.choice(n_new, 256, replace=False):
        assert got[s] == sst.select_one(samples[s], old, oc, act, r, rho), s
    print("large: kept %d of %d, deactivated %d" % (keep.sum(), n_new, deact.sum()))


def test_device_path_equals_host_path():
    old, oc, act, new, nc = _case(5, 1500, 900)
    kh, dh = vine.sst_prune(old, oc, act, new, nc, 3.0, 1.5)
    d = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(d)
    kd, dd = vine.sst_prune(t(old), t(oc), t(act), t(new), t(nc), 3.0, 1.5)
    sh = vine.sst_select(old, oc, act, new, 3.0, 1.5)
    sd = vine.sst_select(t(old), t(oc), t(act), t(new), 3.0, 1.5)
    torch.cuda.synchronize()
    assert np.array_equal(kd.cpu().numpy(), kh) and np.array_equal(dd.cpu().numpy(), dh)
    assert np.array_equal(sd.cpu().numpy(), sh)


def test_degenerate_radii_and_inactive_trees():
    old, oc, act, new, nc = _case(8, 200, 100)
    keep, deact = vine.sst_prune(old, oc, act, new, nc, 0.0, 1.5)
    assert np.array_equal(keep, np.isfinite(nc).astype(np.uint8)) and not deact.any()
    keep, deact = vine.sst_prune(old, oc, act, new, nc, 1e6, 1.5)
    ok, od = sst.prune(old, oc, act, new, nc, 1e6, 1.5)
    assert np.array_equal(keep, ok) and np.array_equal(deact, od) and keep.sum() <= 1
    keep, deact = vine.sst_prune(old, oc, np.zeros_like(act), new, nc, 3.0, 1.5)
    ok, _ = sst.prune(old, oc, np.zeros_like(act), new, nc, 3.0, 1.5)
    assert np.array_equal(keep, ok) and not deact.any()
    assert np.all(vine.sst_select(old, oc, np.zeros_like(act), new, 3.0, 1.5) == -1)
    with pytest.raises(vine.VineError):
        vine.sst_prune(old, oc, act, new, nc, -1.0, 1.5)
    with pytest.raises(vine.VineError):
        vine.sst_select(old, oc, act, new, float("nan"), 1.5)
