"""Pins of the oracle's adjoint (implicit differentiation at the equilibrium
of the last growth step) against central finite differences of re-solved
equilibria: each +-h solve starts from the equilibrium with the design
parameter moved and is converged to 1e-13.  Derivatives whose two solves
differ in contact set, or in the piece of the piecewise model a joint sits on
(sPAM table interval, wrinkling onset), straddle a kink of the model and are
excluded and counted."""
import numpy as np
import pytest

import oracle
from paper_2509_15180_gb300 import scenes

# Steps: at 1e-13 the re-solved equilibria carry ~1e-14 m of solver noise, so
# the steps are chosen where truncation (h^2) and noise (1/h) errors are both
# below 1e-7 of the derivative: 0.1 Pa on pressures of kPa, 1e-4 link.
H_P = 0.1    # Pa
H_S = 1e-4   # link units


def _scene():
    sc, goals = scenes.robustness_batch(n_designs=6, n_perturb=2, n_links=30, box=0.45, n_circ=8, n_box=8)
    # FD steps of 1e-3 Pa and 1e-6 link are below float32 resolution: widen
    sc = {k: (v.astype(np.float64) if v.dtype == np.float32 else v) for k, v in sc.items()}
    return sc, goals.astype(np.float64)


def _tip_cost(orc, i, th, l, goal):
    px, py, _ = orc.poses(i, th, l)
    return float(np.hypot(px[-1] - goal[0], py[-1] - goal[1]))


def _contacts(orc, i, th, l):
    return orc.gaps(i, th, l) < 0.0


def _pieces(orc, sc, i, th, P):
    """Which piece of the piecewise model each joint sits on: the sPAM table
    interval of every covered joint (the force table is piecewise linear in
    strain) and the wrinkling regime (ramp below theta_c, Sec. 3.2).  A
    central difference across a piece boundary straddles a kink."""
    tabs = {t[0]: t for t in orc.tables()}
    d = 2.0 * float(sc["radius"][i]) + P.R_act
    ls = float(sc["l_seg"][i])
    out = [tuple(np.abs(th) > 2.0 * np.arcsin(P.eps_crit))]
    for a in range(int(sc["act_ptr"][i]), int(sc["act_ptr"][i + 1])):
        l0, lo, hi, f = tabs[float(sc["act_l0"][a])]
        hk = (hi - lo) / (len(f) - 1)
        eps = float(sc["act_side"][a]) * d * th / ls
        out.append(tuple(np.floor((eps - lo) / hk).astype(int)))
    return out


def _path_cost(orc, i, th, l, path):
    px, py, _ = orc.poses(i, th, l)
    q = np.asarray(path, np.float64)[: th.size]
    return float(np.mean((px[1:] - q[:, 0]) ** 2 + (py[1:] - q[:, 1]) ** 2))


def _fd(sc, i, key, a_glob, h, th0, l0, goal, P, cost=_tip_cost):
    vals, sets = [], []
    for sgn in (1.0, -1.0):
        mod = dict(sc)
        mod[key] = sc[key].copy()
        mod[key][a_glob] += sgn * h
        orc = oracle.Oracle(mod, P)
        th, l, it, r, st = orc.solve(i, th0, l0)
        if st != 0:
            return None, None
        vals.append(cost(orc, i, th, l, goal))
        sets.append((_contacts(orc, i, th, l), _pieces(orc, mod, i, th, P)))
    same = np.array_equal(sets[0][0], sets[1][0]) and sets[0][1] == sets[1][1]
    return (vals[0] - vals[1]) / (2.0 * h), same


def test_adjoint_matches_central_differences():
    sc, goals = _scene()
    P = oracle.default_params(tol=1e-13)
    orc = oracle.Oracle(sc, oracle.default_params(tol=1e-12))
    st = orc.new_state()
    orc.run(st, 30, threads=8)
    orc13 = oracle.Oracle(sc, P)
    checked = excluded = 0
    worst = 0.0
    rows = []
    for i in range(sc["n_links"].size):
        a0, a1 = int(sc["act_ptr"][i]), int(sc["act_ptr"][i + 1])
        if a1 == a0 or st["status"][i] != 0:
            continue
        th, l, _, _, s13 = orc13.solve(i, orc.theta_of(st, i), st["l"][i])
        assert s13 == 0
        cost, dP, dB, dE, rc = orc13.grad(i, th, l, goals[i])
        assert rc == 0
        assert abs(cost - _tip_cost(orc13, i, th, l, goals[i])) < 1e-15
        for key, h, adj in (("act_pressure", H_P, dP), ("act_begin", H_S, dB), ("act_end", H_S, dE)):
            for a in range(a1 - a0):
                f, ok = _fd(sc, i, key, a0 + a, h, th, l, goals[i], P)
                if f is None or not ok:
                    excluded += 1
                    continue
                rows.append((key, i, a, adj[a], f))
    # each kind of derivative against the largest of its kind in the batch
    # (some are ~0: an actuator whose moment barely reaches the tip)
    for kind in ("act_pressure", "act_begin", "act_end"):
        sel = [r for r in rows if r[0] == kind]
        scale = max(abs(r[4]) for r in sel)
        for (_, i, a, adj, f) in sel:
            err = abs(adj - f) / scale
            worst = max(worst, err)
            assert err < 1e-5, (i, kind, a, adj, f)
            checked += 1
    print("adjoint vs FD: %d derivatives checked, %d excluded (contact set or model piece changed), worst %.2e"
          % (checked, excluded, worst))
    assert checked >= 15


def test_adjoint_pressure_derivative_is_linear_response():
    """Free space: each joint balances M(theta) = sum of actuator moments, so
    the tip moves by d p_N / d P_a = sum_j (z x (p_N - p_j)) dtheta_j/dP_a
    with dtheta_j/dP_a = c_aj s f d / (dM/dtheta - d tau/dtheta) per joint
    (the Hessian is diagonal without contacts)."""
    sc, goals = _scene()
    for k in ("obs_cx", "obs_cy", "obs_a", "obs_b"):
        sc[k] = np.zeros(0)
    sc["obs_kind"] = np.zeros(0, np.uint8)
    sc["obs_ptr"] = np.zeros_like(sc["obs_ptr"])
    orc = oracle.Oracle(sc, oracle.default_params(tol=1e-13))
    st = orc.new_state()
    orc.run(st, 30, threads=8)
    done = 0
    for i in range(sc["n_links"].size):
        a0, a1 = int(sc["act_ptr"][i]), int(sc["act_ptr"][i + 1])
        if a1 == a0:
            continue
        th, l = orc.theta_of(st, i), st["l"][i]
        cost, dP, _, _, rc = orc.grad(i, th, l, goals[i])
        assert rc == 0
        _, g, H = orc.energy(i, th, l)
        Hx = orc.hessian_exact(i, th, l)
        # no contact: the exact Hessian is diagonal in the joint angles
        off = Hx[:-1, :-1] - np.diag(np.diag(Hx[:-1, :-1]))
        assert np.max(np.abs(off)) == 0.0
        px, py, _ = orc.poses(i, th, l)
        e = np.array([px[-1] - goals[i][0], py[-1] - goals[i][1]]) / cost
        N = th.size
        lever = np.stack([-(py[-1] - py[:N]), px[-1] - px[:N]], axis=1)  # z x (p_N - p_j)
        for a in range(a1 - a0):
            # d g_j / d P_a by a finite difference of the gradient alone (the
            # state is held fixed): the actuator moment is linear in P_a
            mod = dict(sc)
            mod["act_pressure"] = sc["act_pressure"].copy()
            mod["act_pressure"][a0 + a] += 1.0
            _, g1, _ = oracle.Oracle(mod).energy(i, th, l)
            dg = (g1 - g)[:N]
            dth = -dg / np.diag(Hx)[:N]
            want = float(e @ (lever.T @ dth))
            assert abs(dP[a] - want) <= 1e-9 * max(abs(want), 1e-12) + 1e-18, (i, a, dP[a], want)
            done += 1
    assert done >= 5


def test_path_cost_adjoint_matches_central_differences():
    """The path cost (1/N) sum_k |p_k - q_k|^2 over the link end points
    against a target path: the adjoint against central differences of
    re-solved equilibria, as for the tip cost."""
    sc, goals = _scene()
    paths = scenes.goal_paths(sc, goals).astype(np.float64)
    off = np.concatenate([[0], np.cumsum(sc["n_links"])])
    P = oracle.default_params(tol=1e-13)
    orc = oracle.Oracle(sc, oracle.default_params(tol=1e-12))
    st = orc.new_state()
    orc.run(st, 30, threads=8)
    orc13 = oracle.Oracle(sc, P)
    rows, excluded = [], 0
    for i in range(sc["n_links"].size):
        a0, a1 = int(sc["act_ptr"][i]), int(sc["act_ptr"][i + 1])
        if a1 == a0 or st["status"][i] != 0:
            continue
        th, l, _, _, s13 = orc13.solve(i, orc.theta_of(st, i), st["l"][i])
        assert s13 == 0
        path = paths[off[i]: off[i + 1]]
        cost, dP, dB, dE, rc = orc13.grad_path(i, th, l, path)
        assert rc == 0
        assert abs(cost - _path_cost(orc13, i, th, l, path)) <= 1e-15 * max(cost, 1e-30)
        for key, h, adj in (("act_pressure", H_P, dP), ("act_begin", H_S, dB), ("act_end", H_S, dE)):
            for a in range(a1 - a0):
                f, ok = _fd(sc, i, key, a0 + a, h, th, l, path, P, cost=_path_cost)
                if f is None or not ok:
                    excluded += 1
                    continue
                rows.append((key, i, a, adj[a], f))
    worst = 0.0
    for kind in ("act_pressure", "act_begin", "act_end"):
        sel = [r for r in rows if r[0] == kind]
        scale = max(abs(r[4]) for r in sel)
        for (_, i, a, adj, f) in sel:
            err = abs(adj - f) / scale
            worst = max(worst, err)
            assert err < 1e-5, (i, kind, a, adj, f)
    print("path-cost adjoint vs FD: %d derivatives, %d excluded, worst %.2e" % (len(rows), excluded, worst))
    assert len(rows) >= 15


def test_path_cost_value_at_arbitrary_states():
    """The cost the adjoint reports is the mean squared distance of the link
    end points to their targets, recomputed from the poses, at states off
    the equilibrium too."""
    sc, goals = _scene()
    orc = oracle.Oracle(sc, oracle.default_params(tol=1e-12))
    st = orc.new_state()
    orc.run(st, 12, threads=8)
    rng = np.random.default_rng(3)
    for i in range(3):
        th, l = orc.theta_of(st, i), float(st["l"][i])
        px, py, _ = orc.poses(i, th, l)
        q = np.stack([px[1:], py[1:]], 1) + rng.normal(0, 0.01, (th.size, 2))
        for _ in range(3):
            tp = th + rng.normal(0, 0.01, th.size)
            c, *_ = orc.grad_path(i, tp, l, q)
            assert abs(c - _path_cost(orc, i, tp, l, q)) <= 1e-14 * c
