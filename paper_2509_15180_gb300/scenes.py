"""Seeded synthetic scenes shaped like the paper's workloads.

This module holds input generation only: random designs and obstacle sets,
no model arithmetic.  Both the CUDA path and the FP64 oracle consume its
output, so that the two start from bit-identical float32 inputs.

The paper's planning environments exist only as figures (Sec. 6.2), so
seeded clutter stands in for them.  Every stream is numpy PCG64 with
seed = 1000 * config + replicate; instances are drawn one after another
from that stream, so the first k instances of a configuration do not depend
on how many are drawn in total.

Scene dictionary (CSR over instances; float32 unless noted):
  n_links[int32 n]   target link count (one link grows per step)
  l_seg, radius, pressure [n]      segment length (m), body radius (m), pressure (Pa)
  base[n, 3]         base x, y (m) and heading (rad)
  act_ptr[int32 n+1], act_begin, act_end (link units, begin < end),
  act_side[int8] (+1 / -1), act_pressure (Pa), act_l0 (sPAM cell length, m)
  obs_ptr[int32 n+1], obs_kind[uint8] (0 circle, 1 axis-aligned box),
  obs_cx, obs_cy (m), obs_a (circle radius or box half-width), obs_b (box half-height)
"""
from __future__ import annotations

import numpy as np

__all__ = ["parity_batch", "design_batch", "uneven_batch", "robustness_batch", "goal_points", "serve_requests",
           "planning_env", "robot_link_steps", "concat", "subset"]


def _rng(config: int, replicate: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * config + replicate))


def _cell_length(l_seg: float) -> float:
    """sPAM cell length: the segment length on the 1 mm fabrication grid (Sec. 4.2)."""
    return round(l_seg * 1000.0) / 1000.0


def _obstacles(rng, n_circ, n_box, r_rng, half_rng, x0, S, keep_out):
    """Obstacles with centres uniform in [x0, x0+S] x [-S/2, S/2]; an obstacle
    whose bounding circle reaches into the keep-out disc around the base is
    redrawn."""
    kinds, cx, cy, a, b = [], [], [], [], []
    for kind, count in ((0, n_circ), (1, n_box)):
        for _ in range(count):
            while True:
                x = rng.uniform(x0, x0 + S)
                y = rng.uniform(-0.5 * S, 0.5 * S)
                if kind == 0:
                    ra = rng.uniform(*r_rng)
                    rb = 0.0
                    reach = ra
                else:
                    ra = rng.uniform(*half_rng)
                    rb = rng.uniform(*half_rng)
                    reach = float(np.hypot(ra, rb))
                if np.hypot(x, y) > reach + keep_out:
                    break
            kinds.append(kind); cx.append(x); cy.append(y); a.append(ra); b.append(rb)
    return kinds, cx, cy, a, b


def _actuators(rng, n_act, n_links, span_rng, p_rng):
    out = []
    for _ in range(n_act):
        span = int(rng.integers(span_rng[0], span_rng[1] + 1))
        span = min(span, n_links)
        begin = int(rng.integers(0, n_links - span + 1))
        side = 1 if rng.random() < 0.5 else -1
        pa = rng.uniform(*p_rng)
        out.append((float(begin), float(begin + span), side, pa))
    return out


def _pack(rows):
    """rows: list of dicts with keys n_links, l_seg, radius, pressure, base, acts, obs."""
    n = len(rows)
    sc = {
        "n_links": np.array([r["n_links"] for r in rows], np.int32),
        "l_seg": np.array([r["l_seg"] for r in rows], np.float32),
        "radius": np.array([r["radius"] for r in rows], np.float32),
        "pressure": np.array([r["pressure"] for r in rows], np.float32),
        "base": np.array([r["base"] for r in rows], np.float32).reshape(n, 3),
    }
    acts = [r["acts"] for r in rows]
    sc["act_ptr"] = np.concatenate([[0], np.cumsum([len(a) for a in acts])]).astype(np.int32)
    flat = [x for a in acts for x in a]
    sc["act_begin"] = np.array([x[0] for x in flat], np.float32)
    sc["act_end"] = np.array([x[1] for x in flat], np.float32)
    sc["act_side"] = np.array([x[2] for x in flat], np.int8)
    sc["act_pressure"] = np.array([x[3] for x in flat], np.float32)
    sc["act_l0"] = np.array([_cell_length(r["l_seg"]) for r in rows for _ in r["acts"]], np.float32)
    obs = [r["obs"] for r in rows]
    sc["obs_ptr"] = np.concatenate([[0], np.cumsum([len(o[0]) for o in obs])]).astype(np.int32)
    sc["obs_kind"] = np.array([k for o in obs for k in o[0]], np.uint8)
    for key, idx in (("obs_cx", 1), ("obs_cy", 2), ("obs_a", 3), ("obs_b", 4)):
        sc[key] = np.array([v for o in obs for v in o[idx]], np.float32)
    return sc


def parity_batch(n_inst: int = 64, replicate: int = 0) -> dict:
    """64 robots x 20 links of 2 cm, R 2.5 cm, P 5 kPa; with probability 1/2 one
    actuator over 5 consecutive links at U[0, 10] kPa; 10 circles of radius
    U[1, 3] cm in a 0.5 m box ahead of the base."""
    rng = _rng(1, replicate)
    rows = []
    for _ in range(n_inst):
        N, ls, R, P = 20, 0.02, 0.025, 5000.0
        acts = _actuators(rng, 1, N, (5, 5), (0.0, 10000.0)) if rng.random() < 0.5 else []
        obs = _obstacles(rng, 10, 0, (0.01, 0.03), None, 0.05, 0.5, R + ls)
        rows.append(dict(n_links=N, l_seg=ls, radius=R, pressure=P, base=(0.0, 0.0, 0.0), acts=acts, obs=obs))
    return _pack(rows)


def design_batch(n_inst: int = 4096, replicate: int = 0) -> dict:
    """4096 robots x 100 links of 1.5 cm, R U[2, 4] cm, P U[2, 10] kPa; 0-6
    actuators over 3-15 links at U[0, 15] kPa; 20 circles (r U[1, 5] cm) and
    20 boxes (sides U[2, 10] cm) in a 1.5 m box."""
    rng = _rng(2, replicate)
    rows = []
    for _ in range(n_inst):
        N, ls = 100, 0.015
        R = rng.uniform(0.02, 0.04)
        P = rng.uniform(2000.0, 10000.0)
        acts = _actuators(rng, int(rng.integers(0, 7)), N, (3, 15), (0.0, 15000.0))
        obs = _obstacles(rng, 20, 20, (0.01, 0.05), (0.01, 0.05), 0.05, 1.5, R + ls)
        rows.append(dict(n_links=N, l_seg=ls, radius=R, pressure=P, base=(0.0, 0.0, 0.0), acts=acts, obs=obs))
    return _pack(rows)


def uneven_batch(n_inst: int = 16384, replicate: int = 0, n_range=(30, 300)) -> dict:
    """Uneven batch: links U{30..300} of U[1, 3] cm, R and P as the design batch, 0-8
    actuators, 5-200 obstacles (half circles, half boxes) in a box whose side
    is the robot's length."""
    rng = _rng(3, replicate)
    rows = []
    for _ in range(n_inst):
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        ls = rng.uniform(0.01, 0.03)
        R = rng.uniform(0.02, 0.04)
        P = rng.uniform(2000.0, 10000.0)
        acts = _actuators(rng, int(rng.integers(0, 9)), N, (3, 15), (0.0, 15000.0))
        n_obs = int(rng.integers(5, 201))
        S = N * ls
        obs = _obstacles(rng, n_obs // 2, n_obs - n_obs // 2, (0.01, 0.05), (0.01, 0.05), 0.05, S, R + ls)
        rows.append(dict(n_links=N, l_seg=ls, radius=R, pressure=P, base=(0.0, 0.0, 0.0), acts=acts, obs=obs))
    return _pack(rows)


def robustness_batch(n_designs: int = 64, n_perturb: int = 1024, replicate: int = 0, n_links: int = 150,
            box: float = 2.25, n_circ: int = 30, n_box: int = 30) -> tuple[dict, np.ndarray]:
    """Robustness batch: designs as the design batch with 150 links and 60 obstacles in
    a 2.25 m box, each perturbed n_perturb times (obstacle centres + N(0, 1 cm),
    actuator endpoints + N(0, 0.5 link), pressures x U[0.95, 1.05]).  Returns
    the scene and one goal point per instance (uniform in the far half of the
    design's box).  The keyword sizes give smaller variants for tests."""
    rng = _rng(4, replicate)
    rows, goals = [], []
    for _ in range(n_designs):
        N, ls = n_links, 0.015
        R = rng.uniform(0.02, 0.04)
        P = rng.uniform(2000.0, 10000.0)
        acts = _actuators(rng, int(rng.integers(0, 7)), N, (3, 15), (0.0, 15000.0))
        S = box
        obs = _obstacles(rng, n_circ, n_box, (0.01, 0.05), (0.01, 0.05), 0.05, S, R + ls)
        goal = (rng.uniform(0.05 + 0.5 * S, 0.05 + S), rng.uniform(-0.5 * S, 0.5 * S))
        for _ in range(n_perturb):
            pk, pcx, pcy, pa, pb = obs
            ncx = list(np.asarray(pcx) + rng.normal(0.0, 0.01, len(pcx)))
            ncy = list(np.asarray(pcy) + rng.normal(0.0, 0.01, len(pcy)))
            pacts = []
            for (b0, e0, sd, pp) in acts:
                b1 = float(np.clip(b0 + rng.normal(0.0, 0.5), 0.0, N - 0.5))
                e1 = float(np.clip(e0 + rng.normal(0.0, 0.5), b1 + 0.5, N))
                pacts.append((b1, e1, sd, pp * rng.uniform(0.95, 1.05)))
            rows.append(dict(n_links=N, l_seg=ls, radius=R, pressure=P, base=(0.0, 0.0, 0.0), acts=pacts,
                             obs=(pk, ncx, ncy, pa, pb)))
            goals.append(goal)
    return _pack(rows), np.array(goals, np.float32)


def goal_points(n_inst: int, box: float, replicate: int = 0) -> np.ndarray:
    """One goal point per instance, uniform in the far half of a box of side
    `box` ahead of the base (as the robustness batch draws them)."""
    rng = _rng(6, replicate)
    gx = rng.uniform(0.05 + 0.5 * box, 0.05 + box, n_inst)
    gy = rng.uniform(-0.5 * box, 0.5 * box, n_inst)
    return np.stack([gx, gy], axis=1).astype(np.float32)


def goal_paths(scene: dict, goals, turn: float = 0.0087) -> np.ndarray:
    """Target points of the link ends for a path cost: per robot its n_links
    points, l_seg apart along an arc that leaves the base toward the robot's
    goal point and turns by `turn` rad per link ([sum n_links, 2] float32,
    robot i's rows in the order of its links)."""
    out = []
    for i, n in enumerate(np.asarray(scene["n_links"])):
        bx, by = float(scene["base"][i][0]), float(scene["base"][i][1])
        ls = float(scene["l_seg"][i])
        phi0 = np.arctan2(float(goals[i][1]) - by, float(goals[i][0]) - bx)
        k = np.arange(1, int(n) + 1)
        phi = phi0 + turn * (k - 0.5)
        out.append(np.stack([bx + ls * np.cumsum(np.cos(phi)), by + ls * np.cumsum(np.sin(phi))], axis=1))
    return np.concatenate(out).astype(np.float32) if out else np.zeros((0, 2), np.float32)


def serve_requests(n_req: int, rate_hz: float = 2000.0, replicate: int = 0, max_inst: int = 256):
    """Poisson request stream for the serving loop: arrival times (s) and, per
    request, a scene of U{1..max_inst} instances drawn as the uneven batch but with
    links U{20..300}."""
    rng = _rng(5, replicate)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_req))
    sizes = rng.integers(1, max_inst + 1, n_req)
    reqs = []
    for k in range(n_req):
        sub = uneven_batch(int(sizes[k]), replicate=5000 + 7919 * replicate + k, n_range=(20, 300))
        reqs.append(sub)
    return t, reqs


def planning_env(kind: str = "channel", replicate: int = 0) -> dict:
    """A planning environment for the batched SST* planner (Sec. 5.2), with
    the paper's robot: R_vine 33.35 mm, P_vine 1.5 psi, 25 mm segments, sPAM
    cells on the 1 mm grid (Sec. 4.2).  The paper's environments exist only
    as figures, so two seeded stand-ins:

    * "channel": a corridor of 2 cm circles (walls 5 cm from the body on
      either side, centres jittered by U[-3, 3] mm) that runs 0.6 m straight
      ahead, bends 90 degrees to the left on a 0.6 m centreline radius and
      runs 0.4 m up; the goal (50 mm radius) is at the corridor's end.
    * "clutter": 40 circles of radius U[2, 6] cm uniform in a 1.4 m box
      ahead of the base (keeping 0.15 m clear around the base); the goal
      (60 mm radius) is at x = 1.4 m, y = U[-0.4, 0.4] m.

    Returns dict(l_seg, radius, pressure, base[3], obs_kind, obs_cx, obs_cy,
    obs_a, obs_b (arrays), goal[2] (m), goal_radius (m), box[4] = x0, x1, y0,
    y1 (m, the sampling region), max_links)."""
    rng = _rng(7, 100 * replicate + (0 if kind == "channel" else 1))
    ls, R, P = 0.025, 0.03335, 1.5 * 6894.757293168
    cx, cy, ca = [], [], []
    if kind == "channel":
        L1, Rc, L2 = 0.6, 0.6, 0.4
        off = R + 0.05 + 0.02
        arc = 0.5 * np.pi * Rc
        total = L1 + arc + L2
        s = 0.0
        while s <= total + 1e-9:
            if s <= L1:
                px, py, tx, ty = s, 0.0, 1.0, 0.0
            elif s <= L1 + arc:
                a = (s - L1) / Rc
                px, py = L1 + Rc * np.sin(a), Rc * (1.0 - np.cos(a))
                tx, ty = np.cos(a), np.sin(a)
            else:
                px, py, tx, ty = L1 + Rc, Rc + (s - L1 - arc), 0.0, 1.0
            nx, ny = -ty, tx
            for side in (1.0, -1.0):
                cx.append(px + side * off * nx + rng.uniform(-0.003, 0.003))
                cy.append(py + side * off * ny + rng.uniform(-0.003, 0.003))
                ca.append(0.02)
            s += 0.045
        goal, goal_r = (L1 + Rc, Rc + L2), 0.05
        box = (-0.1, 1.4, -0.3, 1.2)
        max_links = int(np.ceil(total / ls)) + 12
    elif kind == "clutter":
        while len(cx) < 40:
            x, y, r = rng.uniform(0.1, 1.5), rng.uniform(-0.7, 0.7), rng.uniform(0.02, 0.06)
            if np.hypot(x, y) > r + 0.15:
                cx.append(x); cy.append(y); ca.append(r)
        goal, goal_r = (1.4, rng.uniform(-0.4, 0.4)), 0.06
        box = (-0.1, 1.6, -0.8, 0.8)
        max_links = 80
    else:
        raise ValueError("planning_env: kind must be 'channel' or 'clutter'")
    n = len(cx)
    return dict(l_seg=ls, radius=R, pressure=P, base=np.zeros(3, np.float32),
                obs_kind=np.zeros(n, np.uint8), obs_cx=np.array(cx, np.float32), obs_cy=np.array(cy, np.float32),
                obs_a=np.array(ca, np.float32), obs_b=np.zeros(n, np.float32),
                goal=np.array(goal, np.float64), goal_radius=goal_r, box=np.array(box, np.float64),
                max_links=max_links)


def robot_link_steps(n_links) -> int:
    """Sum over steps of the links present: N (N + 1) / 2 per instance grown from one link."""
    n = np.asarray(n_links, dtype=np.int64)
    return int((n * (n + 1) // 2).sum())


def subset(scene: dict, idx) -> dict:
    """Scene restricted to the instances idx (in that order)."""
    idx = np.asarray(idx, dtype=np.int64)
    out = {k: np.asarray(scene[k])[idx] for k in ("n_links", "l_seg", "radius", "pressure", "base")}
    for pre, ptr in (("act", "act_ptr"), ("obs", "obs_ptr")):
        p = np.asarray(scene[ptr])
        cnt = p[idx + 1] - p[idx]
        out[ptr] = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
        sel = np.concatenate([np.arange(p[i], p[i + 1]) for i in idx]) if len(idx) else np.zeros(0, np.int64)
        sel = sel.astype(np.int64)
        for k in scene:
            if k.startswith(pre + "_") and k != ptr:
                out[k] = np.asarray(scene[k])[sel]
    return out


def concat(scenes) -> dict:
    """Concatenate scenes instance-wise."""
    out = {}
    for k in ("n_links", "l_seg", "radius", "pressure", "base"):
        out[k] = np.concatenate([s[k] for s in scenes])
    for pre, ptr in (("act", "act_ptr"), ("obs", "obs_ptr")):
        ptrs, base = [np.zeros(1, np.int32)], 0
        for s in scenes:
            ptrs.append(np.asarray(s[ptr][1:], np.int64) + base)
            base += int(s[ptr][-1])
        out[ptr] = np.concatenate(ptrs).astype(np.int32)
        for k in scenes[0]:
            if k.startswith(pre + "_") and k != ptr:
                out[k] = np.concatenate([s[k] for s in scenes])
    return out


# ---------------------------------------------------------------------------
# Analysis workloads (Sec. 6.3, 6.4).  The paper's environments and designs
# exist only as figures, so seeded stand-ins with the paper's robot.
# ---------------------------------------------------------------------------
_PAPER_ROBOT = dict(l_seg=0.025, radius=0.03335, pressure=1.5 * 6894.757293168)


def nominal_design(replicate: int = 0) -> dict:
    """A nominal design in a cluttered environment (robustness study): the
    paper's robot, 64 links, two sPAM actuators ([6, 14) pulling to +1 at
    40 kPa, [30, 38) pulling to -1 at 35 kPa), 14 circles of radius
    U[3, 6] cm in [0.2, 1.5] x [-0.5, 0.5] m (0.15 m clear of the base).
    Returns a one-robot scene."""
    rng = _rng(8, replicate)
    cx, cy, ca = [], [], []
    while len(cx) < 14:
        x, y, r = rng.uniform(0.2, 1.5), rng.uniform(-0.5, 0.5), rng.uniform(0.03, 0.06)
        if np.hypot(x, y) - r > 0.15:
            cx.append(x); cy.append(y); ca.append(r)
    row = dict(n_links=64, base=(0.0, 0.0, 0.0), acts=[(6.0, 14.0, 1, 40e3), (30.0, 38.0, -1, 35e3)],
               obs=([0] * len(cx), cx, cy, ca, [0.0] * len(cx)), **_PAPER_ROBOT)
    return _pack([row])


def robustness_sweep(nominal: dict, levels, trials: int = 1000, kind: str = "obstacles", replicate: int = 0):
    """Perturbed copies of a one-robot scene, `trials` per uncertainty level
    (Sec. 6.3; levels as fractions, e.g. 0.05 = 5 %).
      kind "obstacles": every obstacle's radius (or half-sizes) scaled by
        (1 + level z) and its centre moved by level x its radius times z
        per coordinate, z ~ N(0, 1) each;
      kind "actuation": every actuator's pressure scaled by (1 + level z)
        and its span length (end - begin) by (1 + level z'), begin kept.
    Returns (scene, level index per robot)."""
    rng = _rng(9, 1000 * replicate + (0 if kind == "obstacles" else 1))
    nom = nominal
    rows, lev = [], []
    a0, a1 = int(nom["act_ptr"][0]), int(nom["act_ptr"][1])
    o0, o1 = int(nom["obs_ptr"][0]), int(nom["obs_ptr"][1])
    kinds = [int(k) for k in nom["obs_kind"][o0:o1]]
    for li, s in enumerate(levels):
        for _ in range(trials):
            cx = np.asarray(nom["obs_cx"][o0:o1], np.float64).copy()
            cy = np.asarray(nom["obs_cy"][o0:o1], np.float64).copy()
            oa = np.asarray(nom["obs_a"][o0:o1], np.float64).copy()
            ob = np.asarray(nom["obs_b"][o0:o1], np.float64).copy()
            pa = np.asarray(nom["act_pressure"][a0:a1], np.float64).copy()
            bg = np.asarray(nom["act_begin"][a0:a1], np.float64).copy()
            en = np.asarray(nom["act_end"][a0:a1], np.float64).copy()
            if kind == "obstacles":
                size = oa.copy()
                scale = np.maximum(1.0 + s * rng.standard_normal(oa.size), 0.2)
                oa *= scale
                ob = np.where(np.asarray(kinds) == 1, ob * scale, ob)
                cx += s * size * rng.standard_normal(cx.size)
                cy += s * size * rng.standard_normal(cy.size)
            else:
                pa *= np.maximum(1.0 + s * rng.standard_normal(pa.size), 0.0)
                span = (en - bg) * np.maximum(1.0 + s * rng.standard_normal(pa.size), 0.1)
                en = np.minimum(bg + span, float(nom["n_links"][0]))
            rows.append(dict(n_links=int(nom["n_links"][0]), l_seg=float(nom["l_seg"][0]),
                             radius=float(nom["radius"][0]), pressure=float(nom["pressure"][0]),
                             base=tuple(float(v) for v in nom["base"][0]),
                             acts=[(bg[k], en[k], int(nom["act_side"][a0 + k]), pa[k]) for k in range(pa.size)],
                             obs=(kinds, list(cx), list(cy), list(oa), list(ob))))
            lev.append(li)
    return _pack(rows), np.asarray(lev, np.int32)


def funnel_rollouts(n_rollouts: int = 50, counts=(0, 8, 16, 32), n_links: int = 48, replicate: int = 0):
    """The funnelling study (Sec. 6.4): per environment (circles of radius
    U[2, 4] cm uniform in [0.25, 1.25] x [-0.2, 0.8] m, `counts` of them,
    0.15 m clear of the base) n_rollouts robots of the paper's body with
    start headings uniform in [-0.3, 0.3] rad and one actuator over links
    [8, 16) pulling to +1 at 15 kPa x (1 + 0.1 z) -- a varied bending
    control biased toward the upper side.  Returns (scene, environment index
    per robot)."""
    rng = _rng(10, replicate)
    rows, env = [], []
    for e, m in enumerate(counts):
        cx, cy, ca = [], [], []
        while len(cx) < m:
            x, y, r = rng.uniform(0.25, 1.25), rng.uniform(-0.2, 0.8), rng.uniform(0.02, 0.04)
            if np.hypot(x, y) - r > 0.15:
                cx.append(x); cy.append(y); ca.append(r)
        heads = rng.uniform(-0.3, 0.3, n_rollouts)
        for h in heads:
            p = 15e3 * (1.0 + 0.1 * rng.standard_normal())
            rows.append(dict(n_links=n_links, base=(0.0, 0.0, float(h)), acts=[(8.0, 16.0, 1, p)],
                             obs=([0] * m, cx, cy, ca, [0.0] * m), **_PAPER_ROBOT))
            env.append(e)
    return _pack(rows), np.asarray(env, np.int32)
