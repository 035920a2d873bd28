"""Batched SST* design planner (Sec. 5, Algorithm 2) on the GPU path.

A tree node is a grown robot: its joint angles and distal length, the tip
pose p in SE(2), the design that produced it (the actuators along its path
from the root) and its cost.  One iteration of Algorithm 2:

1. sample: B sample poses (seeded, uniform over the environment's box) pick
   the nodes to expand with ``vine_sst_select`` (best near: the cheapest
   active node within the current radius of the sample, else the nearest);
2. sample-action: per expansion a duration of T growth steps (one link per
   step) and a bending control -- none, or one sPAM actuator over the T new
   links with a pressure and a cell length from discrete sets (Sec. 4.2)
   and a side;
3. propagate: one batch of B robots, each loaded with its parent's state
   (``vine_set_state``) and design plus the new actuator, grown T links
   (``vine_simulate``: T steps of the equilibrium growth step);
4. prune: ``vine_sst_prune`` of the resulting tip poses against the active
   tree (keep the cheapest of overlapping states);
5. insert the kept states, deactivate the tree nodes they displace, test
   the goal, and shrink the radius on the schedule of Algorithm 2.

Readings (Sec. 5.1-5.2 leave these open):
* cost = number of actuators on the path + links / max_links: the actuator
  count, with path length as the tie-breaker (a fraction below 1);
* SE(2) metric in millimetres and radians with rho = 100 mm per radian, so
  that r_init = 60 weighs 0.6 rad of heading like 60 mm of position;
* the reverse-tree heuristic (Sec. 5.1) is not used: the paper finds it
  brings no gain (its "No Geo" column), and it needs a third-party planner;
* the schedule's d and l are the dimensions of the tip pose (3) and of the
  bending control (2: pressure and cell length); its iteration count is
  rounded up;
* an expansion whose growth does not converge, or whose tip leaves the
  environment's box, yields no state.

The tree is kept on the host (numpy); every sweep over it, and every growth
step, runs in the library's kernels.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import vine


@dataclass
class PlanConfig:
    batch: int = 1024                    # B: expansions per iteration
    t_range: tuple = (5, 20)             # growth steps per expansion, inclusive
    p_straight: float = 0.3              # probability of an expansion without an actuator
    pressures: tuple = (10e3, 20e3, 40e3, 80e3)  # actuator pressures (Pa)
    cell_lengths: tuple = (0.020, 0.025, 0.030)  # sPAM cell lengths l_0 (m, 1 mm grid)
    r_init: float = 60.0                 # pruning radius (mm + rho rad)
    alpha: float = 0.8                   # radius decay
    sst_iter0: int = 7
    dim_state: int = 3
    dim_control: int = 2
    rho: float = 100.0                   # mm per rad in the SE(2) metric
    seed: int = 0
    params: vine.vine_params | None = None   # None: defaults with two-warp teams (see Planner)


def next_update_iter(i: int, j: int, cfg: PlanConfig) -> int:
    """The radius schedule of Algorithm 2: the iteration of the next radius
    update after the update at iteration i, with j updates so far."""
    return i + int(math.ceil(cfg.sst_iter0 * (1.0 + math.log2(j)) *
                             cfg.alpha ** (-(cfg.dim_state + cfg.dim_control + 1) * j)))


def wrap_angle(phi):
    """Headings to [-pi, pi]."""
    return (np.asarray(phi, np.float64) + np.pi) % (2.0 * np.pi) - np.pi


def node_cost(n_act, n_links, max_links):
    """Actuator count with the robot's length as the tie-breaker."""
    return np.asarray(n_act, np.float64) + np.asarray(n_links, np.float64) / float(max_links)


def sample_actions(rng: np.random.Generator, n: int, cfg: PlanConfig) -> dict:
    """Per expansion: steps T, actuated flag, pressure (Pa), cell length (m),
    side (+1 / -1)."""
    T = rng.integers(cfg.t_range[0], cfg.t_range[1] + 1, n).astype(np.int32)
    act = rng.random(n) >= cfg.p_straight
    pres = np.asarray(cfg.pressures, np.float64)[rng.integers(0, len(cfg.pressures), n)]
    l0 = np.asarray(cfg.cell_lengths, np.float64)[rng.integers(0, len(cfg.cell_lengths), n)]
    side = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    return dict(T=T, actuated=act, pressure=pres, l0=l0, side=side)


def expansion_scene(env: dict, parents_n: np.ndarray, chains: list, actions: dict, max_links: int):
    """The batch that propagates the expansions: robot b has its parent's
    links plus T_b (at most max_links), the parent's actuators plus the new
    one over the new links, and the environment's obstacles.  Returns the
    scene and every robot's actuator list."""
    n = len(parents_n)
    n_links = np.minimum(parents_n + actions["T"], max_links).astype(np.int32)
    acts = []
    for b in range(n):
        a = list(chains[b])
        if actions["actuated"][b] and n_links[b] > parents_n[b]:
            a.append((float(parents_n[b]), float(n_links[b]), int(actions["side"][b]), float(actions["pressure"][b]),
                      float(actions["l0"][b])))
        acts.append(a)
    flat = [x for a in acts for x in a]
    n_obs = len(env["obs_cx"])
    sc = dict(
        n_links=np.maximum(n_links, 1),
        l_seg=np.full(n, env["l_seg"], np.float32),
        radius=np.full(n, env["radius"], np.float32),
        pressure=np.full(n, env["pressure"], np.float32),
        base=np.tile(np.asarray(env["base"], np.float32), (n, 1)),
        act_ptr=np.concatenate([[0], np.cumsum([len(a) for a in acts])]).astype(np.int32),
        act_begin=np.array([x[0] for x in flat], np.float32),
        act_end=np.array([x[1] for x in flat], np.float32),
        act_side=np.array([x[2] for x in flat], np.int8),
        act_pressure=np.array([x[3] for x in flat], np.float32),
        act_l0=np.array([x[4] for x in flat], np.float32),
        obs_ptr=(np.arange(n + 1) * n_obs).astype(np.int32),
        obs_kind=np.tile(env["obs_kind"], n),
        obs_cx=np.tile(env["obs_cx"], n),
        obs_cy=np.tile(env["obs_cy"], n),
        obs_a=np.tile(env["obs_a"], n),
        obs_b=np.tile(env["obs_b"], n),
    )
    return sc, acts


class Planner:
    """Batched SST* over one environment (see the module docstring)."""

    def __init__(self, env: dict, config: PlanConfig | None = None):
        self.env = env
        self.cfg = config or PlanConfig()
        # the expansion batches are uniform and short, so their launches end
        # with their slowest robots: two-warp teams shorten those (measured:
        # 75 ms per iteration against 94 with one warp per robot)
        if self.cfg.params is not None:
            self.params = self.cfg.params
        else:
            self.params = vine.vine_params_default()
            self.params.threads_per_robot = 64
        self.rng = np.random.default_rng(self.cfg.seed)
        self.max_links = int(env["max_links"])
        cap = 1024
        self.pose = np.zeros((cap, 3), np.float32)   # tip x, y (mm), heading (rad)
        self.cost = np.zeros(cap, np.float64)
        self.active = np.zeros(cap, np.uint8)
        self.parent = np.full(cap, -1, np.int64)
        self.n_links = np.zeros(cap, np.int32)
        self.n_act = np.zeros(cap, np.int32)
        self.theta: list = []                        # per node: joint angles (float32)
        self.l_last = np.zeros(cap, np.float32)
        self.chain: list = []                        # per node: actuators on its path
        self.size = 0
        b = env["base"]
        self._insert(np.array([[1000.0 * b[0], 1000.0 * b[1], wrap_angle(b[2])]], np.float32), np.zeros(1),
                     np.array([-1]), np.zeros(1, np.int32), np.zeros(1, np.int32), [np.zeros(0, np.float32)],
                     np.zeros(1, np.float32), [()])
        self.radius = float(self.cfg.r_init)
        self.i = 1
        self.j = 1
        self.next_update = self.cfg.sst_iter0
        self.goal_nodes: list = []
        self.history: list = []

    # -- tree storage -------------------------------------------------------
    def _grow(self, need: int):
        cap = self.pose.shape[0]
        if need <= cap:
            return
        new = max(need, 2 * cap)
        for k in ("pose", "cost", "active", "parent", "n_links", "n_act", "l_last"):
            a = getattr(self, k)
            b = np.zeros((new,) + a.shape[1:], a.dtype)
            if k == "parent":
                b[:] = -1
            b[:cap] = a
            setattr(self, k, b)

    def _insert(self, pose, cost, parent, n_links, n_act, theta, l_last, chain):
        m = len(cost)
        self._grow(self.size + m)
        s = slice(self.size, self.size + m)
        self.pose[s] = pose
        self.cost[s] = cost
        self.active[s] = 1
        self.parent[s] = parent
        self.n_links[s] = n_links
        self.n_act[s] = n_act
        self.l_last[s] = l_last
        self.theta.extend(theta)
        self.chain.extend(chain)
        ids = np.arange(self.size, self.size + m)
        self.size += m
        return ids

    # -- one iteration of Algorithm 2 ----------------------------------------
    def step(self) -> dict:
        cfg, env = self.cfg, self.env
        t0 = time.perf_counter()
        B, M = cfg.batch, self.size
        x0, x1, y0, y1 = (float(v) * 1000.0 for v in env["box"])
        samples = np.stack([self.rng.uniform(x0, x1, B), self.rng.uniform(y0, y1, B),
                            self.rng.uniform(-np.pi, np.pi, B)], 1).astype(np.float32)
        par = vine.sst_select(self.pose[:M], self.cost[:M], self.active[:M], samples, self.radius, cfg.rho)
        par = par[par >= 0].astype(np.int64)
        par = par[self.n_links[par] < self.max_links]
        t1 = time.perf_counter()
        out = dict(iteration=self.i, radius=self.radius, expanded=int(par.size), kept=0, deactivated=0,
                   tree=self.size, goal=False)
        if par.size == 0:
            self._advance()
            out.update(t_select=t1 - t0, t_sim=0.0, t_prune=0.0, t_host=0.0)
            self.history.append(out)
            return out
        acts = sample_actions(self.rng, par.size, cfg)
        pn = self.n_links[par]
        sc, chains = expansion_scene(env, pn, [self.chain[p] for p in par], acts, self.max_links)
        batch = vine.Batch(sc, self.params)
        try:
            offs = batch.offsets
            th = np.zeros(max(batch.total_links, 1), np.float32)
            for b, p in enumerate(par):
                th[offs[b]: offs[b] + pn[b]] = self.theta[p]
            batch.set_state(pn, th, self.l_last[par])
            t2 = time.perf_counter()
            batch.simulate()
            st = batch.state()
        finally:
            batch.close()
        t3 = time.perf_counter()
        N = st["N"]
        ok = (st["status"] == 0) & (N == sc["n_links"])
        heads = st["pose"][np.array([offs[b] + max(int(N[b]), 1) - 1 for b in range(len(N))]), 2]
        tip = st["tip"].astype(np.float64) * 1000.0
        inside = (tip[:, 0] >= x0) & (tip[:, 0] <= x1) & (tip[:, 1] >= y0) & (tip[:, 1] <= y1)
        ok &= inside
        new_pose = np.stack([tip[:, 0], tip[:, 1], wrap_angle(heads)], 1).astype(np.float32)
        n_act = np.array([len(c) for c in chains], np.int32)
        new_cost = node_cost(n_act, N, self.max_links)
        new_cost[~ok] = np.nan
        t4 = time.perf_counter()
        keep, deact = vine.sst_prune(self.pose[:M], self.cost[:M], self.active[:M], new_pose, new_cost,
                                     self.radius, cfg.rho)
        t5 = time.perf_counter()
        self.active[:M][deact != 0] = 0
        k = np.nonzero(keep)[0]
        if k.size:
            ids = self._insert(new_pose[k], new_cost[k], par[k], N[k], n_act[k],
                               [st["theta"][offs[b]: offs[b] + N[b]].copy() for b in k],
                               st["l"][k], [tuple(chains[b]) for b in k])
            g = np.asarray(env["goal"], np.float64) * 1000.0
            d = np.hypot(new_pose[k, 0] - g[0], new_pose[k, 1] - g[1])
            hit = ids[d <= 1000.0 * float(env["goal_radius"])]
            self.goal_nodes.extend(int(h) for h in hit)
            out["goal"] = bool(hit.size)
        out.update(kept=int(k.size), deactivated=int(deact.sum()), tree=self.size, t_select=t1 - t0,
                   t_build=t2 - t1, t_sim=t3 - t2, t_prune=t5 - t4, t_host=(t4 - t3) + (time.perf_counter() - t5),
                   robot_link_steps=int(((N - pn) * (N + pn + 1) // 2)[st["status"] == 0].sum()))
        self.history.append(out)
        self._advance()
        return out

    def _advance(self):
        if self.i == self.next_update:
            self.radius *= self.cfg.alpha
            self.j += 1
            self.next_update = next_update_iter(self.i, self.j, self.cfg)
        self.i += 1

    def run(self, max_iters: int, stop_at_goal: bool = True) -> list:
        for _ in range(max_iters):
            r = self.step()
            if stop_at_goal and r["goal"]:
                break
        return self.history

    # -- solutions -------------------------------------------------------------
    def best_goal(self):
        """The cheapest node that reached the goal region, or None."""
        if not self.goal_nodes:
            return None
        g = np.array(self.goal_nodes)
        return int(g[np.lexsort((g, self.cost[g]))[0]])

    def path(self, node: int) -> list:
        """Nodes from the root to `node`."""
        out = []
        while node >= 0:
            out.append(int(node))
            node = int(self.parent[node])
        return out[::-1]

    def design_scene(self, node: int) -> dict:
        """The node's design as a one-robot scene grown from nothing: its
        actuators, its links and the environment's obstacles (grow it with
        the planner's `params` to reproduce the node bitwise)."""
        chain = list(self.chain[node])
        n_obs = len(self.env["obs_cx"])
        env = self.env
        return dict(
            n_links=np.array([max(int(self.n_links[node]), 1)], np.int32),
            l_seg=np.array([env["l_seg"]], np.float32), radius=np.array([env["radius"]], np.float32),
            pressure=np.array([env["pressure"]], np.float32), base=np.asarray(env["base"], np.float32).reshape(1, 3),
            act_ptr=np.array([0, len(chain)], np.int32),
            act_begin=np.array([c[0] for c in chain], np.float32), act_end=np.array([c[1] for c in chain], np.float32),
            act_side=np.array([c[2] for c in chain], np.int8), act_pressure=np.array([c[3] for c in chain], np.float32),
            act_l0=np.array([c[4] for c in chain], np.float32),
            obs_ptr=np.array([0, n_obs], np.int32), obs_kind=env["obs_kind"].copy(), obs_cx=env["obs_cx"].copy(),
            obs_cy=env["obs_cy"].copy(), obs_a=env["obs_a"].copy(), obs_b=env["obs_b"].copy())
