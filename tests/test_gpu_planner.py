"""The batched SST* planner (Algorithm 2) end to end on the GPU: tree
invariants after several iterations, and every stored node reproduced
bitwise by growing its design from nothing (propagation from stored states
equals growth in one piece)."""
import numpy as np
import pytest

from oracle import sst

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import planner, scenes, vine  # noqa: E402


def _run(kind, iters, batch=256, seed=1):
    p = planner.Planner(scenes.planning_env(kind), planner.PlanConfig(batch=batch, seed=seed))
    hist = p.run(iters, stop_at_goal=False)
    return p, hist


def test_tree_invariants_channel():
    p, hist = _run("channel", 8)
    M = p.size
    assert M > 1 and sum(h["kept"] for h in hist) == M - 1
    act = np.nonzero(p.active[:M])[0]
    # active nodes are pairwise at least the current radius apart (the radius
    # only shrinks, so every insertion kept them so)
    r2 = np.float32(np.float32(p.radius) * np.float32(p.radius))
    P = p.pose[act]
    for a in range(len(act)):
        d2 = sst._dist2_rows(P[a], P[a + 1:], p.cfg.rho)
        assert np.all(d2 >= r2), (act[a], np.min(d2))
    for k in range(1, M):
        par = p.parent[k]
        assert 0 <= par < k
        assert p.n_links[k] > p.n_links[par]
        assert p.n_act[k] in (p.n_act[par], p.n_act[par] + 1)
        assert p.cost[k] == planner.node_cost(p.n_act[k], p.n_links[k], p.max_links)
        assert len(p.theta[k]) == p.n_links[k]
    print("channel: %d nodes, %d active, radius %.1f, expansions %s" % (M, len(act), p.radius,
                                                                      [h["expanded"] for h in hist]))


def test_nodes_replay_bitwise_from_their_designs():
    p, _ = _run("clutter", 5, batch=192, seed=2)
    rng = np.random.default_rng(0)
    deep = [k for k in range(1, p.size) if len(p.path(k)) >= 3]
    pick = list(rng.choice(deep, min(12, len(deep)), replace=False)) if deep else []
    pick += list(rng.choice(np.arange(1, p.size), 12, replace=False))
    scs = [p.design_scene(int(k)) for k in pick]
    b = vine.Batch(scenes.concat(scs), p.params)
    b.simulate()
    st = b.state()
    for j, k in enumerate(pick):
        assert st["status"][j] == 0 and st["N"][j] == p.n_links[k]
        assert np.array_equal(b.theta_of(st, j), p.theta[k]), k
        assert st["l"][j] == p.l_last[k]
        tip = st["tip"][j].astype(np.float64) * 1000.0
        head = planner.wrap_angle(b.pose_of(st, j)[-1, 2])
        assert np.array_equal(np.array([tip[0], tip[1], head], np.float32), p.pose[k]), k
    b.close()
    print("replayed %d nodes (%d at depth >= 2)" % (len(pick), min(12, len(deep))))
