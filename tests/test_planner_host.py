"""Host logic of the batched SST* planner (Algorithm 2): the radius
schedule, costs, action sampling, the expansion batch's layout and the tree
bookkeeping, on the CPU (no kernel runs here)."""
import math

import numpy as np

from paper_2509_15180_gb300 import build

build.build()
from paper_2509_15180_gb300 import planner, scenes  # noqa: E402


def test_radius_schedule_hand_values():
    cfg = planner.PlanConfig()
    # first update at sst_iter0 = 7; then i + ceil(7 (1 + log2 j) 0.8^(-6 j))
    assert planner.next_update_iter(7, 2, cfg) == 7 + 204        # 14 / 0.8^12 = 203.73
    assert planner.next_update_iter(211, 3, cfg) == 211 + 1005   # 7 (1 + log2 3) / 0.8^18 = 1004.47
    p = planner.Planner(scenes.planning_env("channel"), cfg)
    radii = []
    for _ in range(220):
        radii.append(p.radius)
        p._advance()
    assert radii[6] == 60.0 and radii[7] == 60.0 * 0.8            # shrinks after iteration 7
    assert radii[210] == 60.0 * 0.8 and math.isclose(radii[211], 60.0 * 0.64)


def test_wrap_and_cost():
    assert np.allclose(planner.wrap_angle([1.5 * np.pi, -np.pi, np.pi, 0.3, -4.0]),
                       [-0.5 * np.pi, -np.pi, -np.pi, 0.3, 2 * np.pi - 4.0])
    assert planner.node_cost(2, 45, 90) == 2.5
    assert np.all(planner.node_cost([0, 1, 3], [89, 0, 10], 90) < [1, 2, 4])


def test_action_sampling_ranges_and_seed():
    cfg = planner.PlanConfig()
    a = planner.sample_actions(np.random.default_rng(3), 20000, cfg)
    b = planner.sample_actions(np.random.default_rng(3), 20000, cfg)
    for k in a:
        assert np.array_equal(a[k], b[k])
    assert a["T"].min() == cfg.t_range[0] and a["T"].max() == cfg.t_range[1]
    assert set(np.unique(a["pressure"])) == set(cfg.pressures)
    assert set(np.unique(a["l0"])) == set(cfg.cell_lengths)
    assert set(np.unique(a["side"])) == {-1, 1}
    assert abs((~a["actuated"]).mean() - cfg.p_straight) < 0.02


def test_expansion_scene_layout():
    env = scenes.planning_env("clutter")
    chains = [(), ((0.0, 7.0, 1, 2e4, 0.025),), ((0.0, 5.0, -1, 1e4, 0.02), (5.0, 12.0, 1, 4e4, 0.03))]
    pn = np.array([0, 7, 78], np.int32)
    acts = dict(T=np.array([6, 9, 10], np.int32), actuated=np.array([True, False, True]),
                pressure=np.array([8e4, 1e4, 2e4]), l0=np.array([0.02, 0.025, 0.03]), side=np.array([-1, 1, 1], np.int8))
    sc, lists = planner.expansion_scene(env, pn, chains, acts, env["max_links"])
    assert sc["n_links"].tolist() == [6, 16, 80]                 # capped at max_links
    assert sc["act_ptr"].tolist() == [0, 1, 2, 5]
    assert sc["act_begin"].tolist() == [0.0, 0.0, 0.0, 5.0, 78.0]
    assert sc["act_end"].tolist() == [6.0, 7.0, 5.0, 12.0, 80.0]
    assert sc["act_side"].tolist() == [-1, 1, -1, 1, 1]
    n_obs = len(env["obs_cx"])
    assert sc["obs_ptr"].tolist() == [0, n_obs, 2 * n_obs, 3 * n_obs]
    assert np.array_equal(sc["obs_cx"][n_obs: 2 * n_obs], env["obs_cx"])
    assert [len(x) for x in lists] == [1, 1, 3]


def test_tree_bookkeeping():
    env = scenes.planning_env("channel")
    p = planner.Planner(env)
    assert p.size == 1 and p.active[0] == 1 and p.parent[0] == -1
    # a chain root -> a -> b, and a sibling c that reached the goal cheaper
    ch_a = ((0.0, 10.0, 1, 4e4, 0.025),)
    ida = p._insert(np.array([[250, 0, 0.1]], np.float32), np.array([1 + 10 / 90]), np.array([0]),
                    np.array([10], np.int32), np.array([1], np.int32), [np.zeros(10, np.float32)],
                    np.array([0.02], np.float32), [ch_a])
    idb = p._insert(np.array([[500, 50, 0.5]], np.float32), np.array([1 + 25 / 90]), ida,
                    np.array([25], np.int32), np.array([1], np.int32), [np.zeros(25, np.float32)],
                    np.array([0.01], np.float32), [ch_a])
    for _ in range(1500):  # storage growth keeps what was there
        p._insert(np.zeros((1, 3), np.float32), np.ones(1), np.array([0]), np.ones(1, np.int32),
                  np.zeros(1, np.int32), [np.zeros(1, np.float32)], np.zeros(1, np.float32), [()])
    assert p.path(int(idb[0])) == [0, int(ida[0]), int(idb[0])]
    assert p.cost[idb[0]] == 1 + 25 / 90 and p.n_links[ida[0]] == 10
    p.goal_nodes = [int(idb[0]), int(ida[0])]
    assert p.best_goal() == int(ida[0])
    d = p.design_scene(int(idb[0]))
    assert d["n_links"].tolist() == [25] and d["act_ptr"].tolist() == [0, 1]
    assert d["act_end"].tolist() == [10.0] and d["obs_ptr"][-1] == len(env["obs_cx"])
