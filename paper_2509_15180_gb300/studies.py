"""The paper's analysis workloads, each one batched launch of the growth
step (Sec. 6.3, 6.4), on seeded stand-ins for its environments.

* Robustness (Sec. 6.3): a nominal design is grown once; its tip is the
  centre of the goal region.  For every uncertainty level, `trials` copies of
  the design are perturbed -- the obstacles (sizes and positions) or the
  actuation (pressures and span lengths) -- and all levels of one kind grow
  together in one vine_simulate.  The success rate of a level is the share
  of its robots that grew to full length and ended with the tip inside the
  goal region.
* Funnelling (Sec. 6.4): rollouts with uniformly spread start headings and a
  varied bending control in environments of rising obstacle density, all in
  one vine_simulate; the k-nearest-neighbour density concentration ratio of
  the end points per environment and k.

The growth runs in libvine.so; the statistics are host code on the returned
tips (analysis.py).
"""
from __future__ import annotations

import time

import numpy as np

from . import analysis, scenes, vine

LEVELS = tuple(round(0.02 * k, 2) for k in range(11))  # 0 .. 20 %


def _grow(sc, params=None, stream=None):
    b = vine.Batch(sc, params, stream=stream)
    t0 = time.perf_counter()
    b.simulate(stream)
    st = b.state(stream)
    wall = time.perf_counter() - t0
    rls = b.stats(stream)["robot_link_steps"]
    b.close()
    return st, wall, rls


def robustness(levels=LEVELS, trials: int = 1000, goal_radius: float = 0.1, replicate: int = 0, params=None,
               stream=None) -> dict:
    """Success rate against uncertainty level for obstacle and actuation
    perturbations of the nominal design (1000 trials per level by
    default)."""
    nom = scenes.nominal_design(replicate)
    st0, _, _ = _grow(nom, params, stream)
    if st0["status"][0] != 0:
        raise RuntimeError("the nominal design did not grow to equilibrium")
    goal = st0["tip"][0].astype(np.float64)
    out = {"goal": goal.tolist(), "goal_radius": goal_radius, "levels": list(levels), "trials": trials}
    for kind in ("obstacles", "actuation"):
        sc, lev = scenes.robustness_sweep(nom, levels, trials, kind, replicate)
        st, wall, rls = _grow(sc, params, stream)
        done = st["status"] == 0
        reach = np.hypot(st["tip"][:, 0] - goal[0], st["tip"][:, 1] - goal[1]) <= goal_radius
        rate = [float(np.mean((done & reach)[lev == k])) for k in range(len(levels))]
        out[kind] = {"success_rate": rate, "robots": int(lev.size), "not_converged": int((~done).sum()),
                     "seconds": wall, "robot_link_steps": int(rls), "tips": st["tip"], "status": st["status"]}
    return out


def funnel(ks=(3, 5, 8, 10), n_rollouts: int = 50, counts=(0, 8, 16, 32), replicate: int = 0, params=None,
           stream=None) -> dict:
    """k-NN density concentration ratio of the rollouts' end points per
    environment (rising obstacle count) and k."""
    sc, env = scenes.funnel_rollouts(n_rollouts, counts, replicate=replicate)
    st, wall, rls = _grow(sc, params, stream)
    done = st["status"] == 0
    ratios = []
    for e in range(len(counts)):
        pts = st["tip"][(env == e) & done]
        ratios.append({int(k): analysis.density_concentration_ratio(pts, int(k)) for k in ks if len(pts) > k})
    return {"obstacles": list(counts), "rollouts": n_rollouts, "ratio": ratios, "not_converged": int((~done).sum()),
            "seconds": wall, "robot_link_steps": int(rls), "tips": st["tip"], "status": st["status"], "env": env}
