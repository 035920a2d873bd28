"""Pins for the oracle's chain energy, gradient and equilibrium solver (CPU only).

Pins used here: finite differences of the oracle's energy (FP64), closed-form
equilibria (straight tube; decoupled free-space joints solved by scalar
bisection; a uniform actuator bends the chain into a regular polygon),
a static free-body balance recomputed from the returned poses with an
independent signed-distance routine, a library optimiser on tiny scenes,
dense boundary sampling for the signed distances, and mirror / rigid-motion
symmetry.
"""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle
from paper_2509_15180_gb300 import scenes

PI = math.pi


def scene_of(rows):
    """rows: list of dict(n, l_seg, R, P, base=(x,y,psi), acts=[(b,e,side,Pa,l0)], obs=[(kind,cx,cy,a,b)])."""
    sc = {"n_links": np.array([r["n"] for r in rows], np.int32),
          "l_seg": np.array([r["l_seg"] for r in rows], np.float32),
          "radius": np.array([r["R"] for r in rows], np.float32),
          "pressure": np.array([r["P"] for r in rows], np.float32),
          "base": np.array([r.get("base", (0.0, 0.0, 0.0)) for r in rows], np.float32)}
    acts = [r.get("acts", []) for r in rows]
    obs = [r.get("obs", []) for r in rows]
    sc["act_ptr"] = np.concatenate([[0], np.cumsum([len(a) for a in acts])]).astype(np.int32)
    fa = [a for aa in acts for a in aa]
    sc["act_begin"] = np.array([a[0] for a in fa], np.float32)
    sc["act_end"] = np.array([a[1] for a in fa], np.float32)
    sc["act_side"] = np.array([a[2] for a in fa], np.int8)
    sc["act_pressure"] = np.array([a[3] for a in fa], np.float32)
    sc["act_l0"] = np.array([a[4] for a in fa], np.float32)
    sc["obs_ptr"] = np.concatenate([[0], np.cumsum([len(o) for o in obs])]).astype(np.int32)
    fo = [o for oo in obs for o in oo]
    sc["obs_kind"] = np.array([o[0] for o in fo], np.uint8)
    for k, j in (("obs_cx", 1), ("obs_cy", 2), ("obs_a", 3), ("obs_b", 4)):
        sc[k] = np.array([o[j] for o in fo], np.float32)
    return sc


def grow(orc, steps):
    st = orc.new_state()
    orc.run(st, steps)
    return st


# ------------------------------------------------------------------ P1
def test_straight_unactuated_stays_straight():
    base = (0.1, -0.2, 0.3)
    sc = scene_of([dict(n=12, l_seg=0.02, R=0.025, P=5000.0, base=base)])
    o = oracle.Oracle(sc)
    st = grow(o, 12)
    th = o.theta_of(st, 0)
    assert st["status"][0] == 0 and st["conv"][0] == 12
    assert np.all(th == 0.0)
    assert st["l"][0] == pytest.approx(float(np.float32(0.02)), rel=1e-15)
    px, py, psi = o.poses(0, th, st["l"][0])
    ls = float(np.float32(0.02))
    b = np.array(base, np.float32).astype(float)
    k = np.arange(13)
    assert np.allclose(px, b[0] + k * ls * math.cos(b[2]), atol=1e-15, rtol=0)
    assert np.allclose(py, b[1] + k * ls * math.sin(b[2]), atol=1e-15, rtol=0)


def test_growth_energy_closed_form():
    sc = scene_of([dict(n=3, l_seg=0.02, R=0.03, P=4000.0)])
    o = oracle.Oracle(sc)
    ls, R, P = [float(np.float32(v)) for v in (0.02, 0.03, 4000.0)]
    kg = PI * P * R * R / (2 * ls)
    for l in (0.0, 0.005, 0.02):
        J, g, _ = o.energy(0, np.zeros(3), l)
        assert J == pytest.approx(15.0 * kg * (ls - l) ** 2, rel=1e-14, abs=1e-18)
        assert g[3] == pytest.approx(-2 * 15.0 * kg * (ls - l), rel=1e-14, abs=1e-18)


# ------------------------------------------------------------------ signed distances
def _sample_boundary(kind, cx, cy, a, b, n=400000):
    if kind == 0:
        t = np.linspace(0, 2 * PI, n, endpoint=False)
        return np.stack([cx + a * np.cos(t), cy + a * np.sin(t)], 1)
    m = n // 4
    s = np.linspace(-1, 1, m)
    return np.concatenate([np.stack([cx + a * s, cy - b + 0 * s], 1), np.stack([cx + a * s, cy + b + 0 * s], 1),
                           np.stack([cx - a + 0 * s, cy + b * s], 1), np.stack([cx + a + 0 * s, cy + b * s], 1)])


@pytest.mark.parametrize("kind", [0, 1])
def test_sdf_vs_dense_boundary_sampling(kind):
    cx, cy, a, b = 0.3, -0.1, 0.04, (0.025 if kind else 0.0)
    sc = scene_of([dict(n=1, l_seg=0.02, R=0.02, P=1000.0, obs=[(kind, cx, cy, a, b)])])
    o = oracle.Oracle(sc)
    cx, cy, a, b = [float(np.float32(v)) for v in (cx, cy, a, b)]
    pts = _sample_boundary(kind, cx, cy, a, b)
    rng = np.random.default_rng(5)
    for _ in range(60):
        x, y = cx + rng.uniform(-0.09, 0.09), cy + rng.uniform(-0.09, 0.09)
        d, nx, ny = o.sdf(0, x, y)
        dist = np.min(np.hypot(pts[:, 0] - x, pts[:, 1] - y))
        inside = (math.hypot(x - cx, y - cy) < a) if kind == 0 else (abs(x - cx) < a and abs(y - cy) < b)
        assert abs(abs(d) - dist) < 2e-6
        assert (d < 0) == inside
        h = 1e-7
        gx = (o.sdf(0, x + h, y)[0] - o.sdf(0, x - h, y)[0]) / (2 * h)
        gy = (o.sdf(0, x, y + h)[0] - o.sdf(0, x, y - h)[0]) / (2 * h)
        if abs(abs(x - cx) - a) > 1e-5 and abs(abs(y - cy) - b) > 1e-5 and abs(
                (abs(x - cx) - a) - (abs(y - cy) - b)) > 1e-5:
            assert nx == pytest.approx(gx, abs=1e-6) and ny == pytest.approx(gy, abs=1e-6)


# ------------------------------------------------------------------ energy derivatives
def contact_scene(n=6, K=2, seed=0):
    rng = np.random.default_rng(seed)
    ls, R = 0.02, 0.025
    obs = [(0, 0.06, 0.045, 0.03, 0.0), (1, 0.10, -0.05, 0.02, 0.015), (0, 0.14, 0.04, 0.01, 0.0)]
    acts = [(0.5, 3.5, 1, 8000.0, 0.02), (2.0, 6.0, -1, 3000.0, 0.02)]
    return scene_of([dict(n=n, l_seg=ls, R=R, P=5000.0, acts=acts, obs=obs)]), rng


def test_gradient_matches_finite_differences():
    sc, rng = contact_scene()
    o = oracle.Oracle(sc)
    for trial in range(6):
        th = rng.normal(0, 0.08, 6)
        l = rng.uniform(0.002, 0.019)
        J, g, _ = o.energy(0, th, l, hessian=False)
        h = 1e-7
        fd = np.zeros(7)
        for k in range(7):
            tp, tm = th.copy(), th.copy()
            lp, lm = l, l
            if k < 6:
                tp[k] += h; tm[k] -= h
            else:
                lp += h; lm -= h
            fd[k] = (o.energy(0, tp, lp, False)[0] - o.energy(0, tm, lm, False)[0]) / (2 * h)
        scale = np.max(np.abs(g))
        assert np.max(np.abs(g - fd)) <= 2e-6 * scale, (g, fd)


def test_hessian_exact_without_contact():
    """Without contact the Gauss-Newton matrix is the exact Hessian: compare with
    finite differences of the gradient."""
    sc = scene_of([dict(n=5, l_seg=0.02, R=0.025, P=5000.0, acts=[(0.3, 4.2, 1, 9000.0, 0.02)])])
    o = oracle.Oracle(sc)
    th = np.array([0.01, 0.03, -0.002, 0.2, 0.05])
    l = 0.013
    _, g, H = o.energy(0, th, l)
    h = 1e-7
    for k in range(6):
        tp, tm = th.copy(), th.copy()
        lp, lm = l, l
        if k < 5:
            tp[k] += h; tm[k] -= h
        else:
            lp += h; lm -= h
        col = (o.energy(0, tp, lp, False)[1] - o.energy(0, tm, lm, False)[1]) / (2 * h)
        assert np.allclose(H[:, k], col, rtol=1e-5, atol=1e-6 * np.abs(H).max())


def test_gauss_newton_contact_rows():
    """With one disc per link, each (link, obstacle) pair is one contact whose
    penetration is minus its gap: H - diag(bending) - growth = kappa sum v v^T
    with v the finite-difference gradient of the penetration."""
    sc, rng = contact_scene()
    P = oracle.default_params(discs_per_link=1)
    o = oracle.Oracle(sc, P)
    th = np.array([0.05, 0.1, -0.05, 0.1, 0.0, -0.1])
    l = 0.015
    gap0 = o.gaps(0, th, l)
    assert (gap0 < 0).sum() >= 2
    _, _, H = o.energy(0, th, l)
    # bending/growth diagonal from a far-away copy of the obstacles
    sc2 = dict(sc)
    sc2["obs_cx"] = sc["obs_cx"] + np.float32(50.0)
    _, _, Hb = oracle.Oracle(sc2, P).energy(0, th, l)
    ls, R, Pv = [float(np.float32(v)) for v in (0.02, 0.025, 5000.0)]
    kc = 160.0 * PI * Pv * R ** 3 / (2 * 0.01 * R * ls)
    h = 1e-8
    V = []
    for (i, ob) in zip(*np.nonzero(gap0 < 0)):
        v = np.zeros(7)
        for k in range(7):
            tp, tm = th.copy(), th.copy()
            lp, lm = l, l
            if k < 6:
                tp[k] += h; tm[k] -= h
            else:
                lp += h; lm -= h
            v[k] = -(o.gaps(0, tp, lp)[i, ob] - o.gaps(0, tm, lm)[i, ob]) / (2 * h)
        V.append(v)
    V = np.array(V)
    ref = Hb + 2 * kc * V.T @ V
    assert np.allclose(H, ref, rtol=1e-6, atol=1e-6 * np.abs(H).max())


@pytest.mark.parametrize("ks", [1, 2])
def test_exact_hessian_matches_finite_differences(ks):
    """The exact Hessian (obstacle curvature and load-stiffness terms of the
    contact penalty included) equals central differences of the gradient."""
    sc, rng = contact_scene()
    o = oracle.Oracle(sc, oracle.default_params(discs_per_link=ks))
    for _ in range(6):
        th = rng.normal(0, 0.08, 6)
        l = rng.uniform(0.002, 0.019)
        H = o.hessian_exact(0, th, l)
        h = 1e-7
        Hf = np.zeros((7, 7))
        for k in range(7):
            tp, tm = th.copy(), th.copy()
            lp, lm = l, l
            if k < 6:
                tp[k] += h; tm[k] -= h
            else:
                lp += h; lm -= h
            Hf[:, k] = (o.energy(0, tp, lp, False)[1] - o.energy(0, tm, lm, False)[1]) / (2 * h)
        assert np.max(np.abs(H - Hf)) <= 1e-7 * np.max(np.abs(Hf))


# ------------------------------------------------------------------ P2 / P3 free space
def _free_joint_balance(o, sc, i, j, lo, hi):
    """Scalar FP64 bisection of M(theta) = sum_a tau_a(theta) at joint j."""
    P = o.P
    R, Pv, ls = [float(sc[k][i]) for k in ("radius", "pressure", "l_seg")]
    d = 2 * R + P.R_act
    tabs = {t[0]: t[1:] for t in o.tables()}
    a0, a1 = sc["act_ptr"][i], sc["act_ptr"][i + 1]

    def f(th):
        m = PI * Pv * R ** 3 * oracle.wrinkle(th, P.eps_crit, energy=False)[0]
        for a in range(a0, a1):
            b, e = float(sc["act_begin"][a]), float(sc["act_end"][a])
            c = max(0.0, min(e, j + 1) - max(b, j))
            if c <= 0:
                continue
            s, Pa, l0 = int(sc["act_side"][a]), float(sc["act_pressure"][a]), float(sc["act_l0"][a])
            lo_, hi_, fk = tabs[l0]
            m -= c * s * Pa * oracle.table_eval(lo_, hi_, fk, s * d * th / ls)[0] * d
        return m

    return optimize.brentq(f, lo, hi, xtol=1e-15, rtol=1e-15)


def test_free_space_decoupled_joints():
    rows = [dict(n=10, l_seg=0.02, R=0.025, P=5000.0,
                 acts=[(2.0, 7.0, 1, 10000.0, 0.02), (5.5, 9.0, -1, 6000.0, 0.02)]),
            dict(n=8, l_seg=0.015, R=0.04, P=2000.0, acts=[(0.0, 8.0, -1, 15000.0, 0.015)]),
            dict(n=8, l_seg=0.015, R=0.02, P=10000.0, acts=[(1.25, 4.75, 1, 1000.0, 0.015)])]
    sc = scene_of(rows)
    o = oracle.Oracle(sc, oracle.default_params(tol=1e-12))
    st = grow(o, 10)
    for i in range(3):
        th = o.theta_of(st, i)
        for j in range(len(th)):
            ref = _free_joint_balance(o, sc, i, j, -1.0, 1.0)
            assert th[j] == pytest.approx(ref, abs=1e-10)


def test_uniform_actuator_regular_polygon():
    """An actuator covering every link bends every joint by the same angle; the
    link start points are then p_n = l_seg sum_{k<n} exp(i (psi_b + (k+1) theta))."""
    sc = scene_of([dict(n=9, l_seg=0.02, R=0.025, P=5000.0, base=(0.0, 0.0, 0.2),
                        acts=[(0.0, 9.0, 1, 7000.0, 0.02)])])
    o = oracle.Oracle(sc, oracle.default_params(tol=1e-12))
    st = grow(o, 9)
    th = o.theta_of(st, 0)
    assert np.allclose(th, th[0], atol=1e-13, rtol=0)
    t0 = _free_joint_balance(o, sc, 0, 0, -1.0, 1.0)
    assert th[0] == pytest.approx(t0, abs=1e-12)
    px, py, _ = o.poses(0, th, st["l"][0])
    ls, pb = float(np.float32(0.02)), float(np.float32(0.2))
    z = np.concatenate([[0], np.cumsum(ls * np.exp(1j * (pb + (np.arange(9) + 1) * t0)))])
    assert np.allclose(px, z.real, atol=1e-13) and np.allclose(py, z.imag, atol=1e-13)


def test_below_threshold_ramp():
    """A weak actuator keeps every joint on the ramp below wrinkling onset,
    where theta = theta_c tau(theta) / M_on; zero pressure gives theta = 0."""
    sc = scene_of([dict(n=6, l_seg=0.02, R=0.03, P=8000.0, acts=[(0.0, 3.0, 1, 150.0, 0.02)]),
                   dict(n=6, l_seg=0.02, R=0.03, P=8000.0, acts=[(0.0, 6.0, 1, 0.0, 0.02)])])
    o = oracle.Oracle(sc, oracle.default_params(tol=1e-12))
    st = grow(o, 6)
    thc = 2 * math.asin(0.01)
    th = o.theta_of(st, 0)
    assert np.all(np.abs(th) <= thc) and th[0] > 0
    R, Pv, ls = [float(np.float32(v)) for v in (0.03, 8000.0, 0.02)]
    d = 2 * R + 0.01718
    lo, hi, fk = o.tables()[0][1:]
    for j in range(3):
        tau = float(np.float32(150.0)) * oracle.table_eval(lo, hi, fk, d * th[j] / ls)[0] * d
        assert th[j] == pytest.approx(thc * tau / (PI * Pv * R ** 3 / 2), rel=1e-10)
    assert np.all(th[3:] == 0.0)
    assert np.all(o.theta_of(st, 1) == 0.0)


# ------------------------------------------------------------------ P6 free-body balance
def _np_sdf(kind, cx, cy, a, b, x, y):
    if kind == 0:
        d = math.hypot(x - cx, y - cy)
        return d - a, ((x - cx) / d, (y - cy) / d)
    dx, dy = x - cx, y - cy
    qx, qy = abs(dx) - a, abs(dy) - b
    sx, sy = math.copysign(1, dx), math.copysign(1, dy)
    if qx > 0 and qy > 0:
        d = math.hypot(qx, qy)
        return d, (sx * qx / d, sy * qy / d)
    if qx > 0 or (qy <= 0 and qx >= qy):
        return qx, (sx, 0.0)
    return qy, (0.0, sy)


def test_static_balance_at_equilibrium():
    """At the returned state every joint balances: w_a M_tot,j equals the moment
    about p_j of the contact forces 2 w_c k_c pen n on all distal discs, and the
    tip force balances growth (forces recomputed here from poses alone)."""
    sc = scenes.parity_batch(24)
    o = oracle.Oracle(sc, oracle.default_params(tol=1e-11))
    st = grow(o, 20)
    checked = 0
    for i in range(sc["n_links"].size):
        th = o.theta_of(st, i)
        N, l = th.size, st["l"][i]
        px, py, psi = o.poses(0 * i + i, th, l)
        R, Pv, ls = [float(sc[k][i]) for k in ("radius", "pressure", "l_seg")]
        kc = 160.0 * PI * Pv * R ** 3 / (2 * 0.01 * R * ls)
        F = []  # (x, y, fx, fy, link, frac)
        for k in range(N):
            L = ls if k < N - 1 else l
            u = (math.cos(psi[k]), math.sin(psi[k]))
            for q in (1, 2):
                x, y = px[k] + q / 2 * L * u[0], py[k] + q / 2 * L * u[1]
                for ob in range(sc["obs_ptr"][i], sc["obs_ptr"][i + 1]):
                    sd, n = _np_sdf(int(sc["obs_kind"][ob]), *[float(sc[c][ob]) for c in
                                                               ("obs_cx", "obs_cy", "obs_a", "obs_b")], x, y)
                    if R - sd > 0:
                        f = 2 * kc * (R - sd)
                        F.append((x, y, f * n[0], f * n[1], k, q / 2))
        if not F:
            continue
        checked += 1
        PR3 = PI * Pv * R ** 3
        d = 2 * R + o.P.R_act
        tabs = {tb[0]: tb[1:] for tb in o.tables()}
        for j in range(N):
            mtot = PR3 * oracle.wrinkle(th[j], o.P.eps_crit, energy=False)[0]
            for a in range(sc["act_ptr"][i], sc["act_ptr"][i + 1]):
                c = max(0.0, min(float(sc["act_end"][a]), j + 1) - max(float(sc["act_begin"][a]), j))
                if c > 0:
                    s_, Pa = int(sc["act_side"][a]), float(sc["act_pressure"][a])
                    lo_, hi_, fk = tabs[float(sc["act_l0"][a])]
                    mtot -= c * s_ * Pa * oracle.table_eval(lo_, hi_, fk, s_ * d * th[j] / ls)[0] * d
            mom = sum((x - px[j]) * fy - (y - py[j]) * fx for (x, y, fx, fy, k, _) in F if k >= j)
            assert abs(160.0 * mtot - mom) <= 1e-7 * 160.0 * PR3 + 1e-7 * abs(mom)
        # tip: growth force balances the contact push along the distal link
        if l < ls:
            u = (math.cos(psi[N - 1]), math.sin(psi[N - 1]))
            push = sum(fr * (fx * u[0] + fy * u[1]) for (x, y, fx, fy, k, fr) in F if k == N - 1)
            kg = PI * Pv * R * R / (2 * ls)
            assert abs(2 * 15.0 * kg * (ls - l) + push) <= 1e-7 * PI * Pv * R * R
    assert checked >= 5


# ------------------------------------------------------------------ P7 brute force
def test_tiny_scene_local_minimum():
    """On tiny scenes a library optimiser started from the same warm start
    finds the same local minimum of the oracle's energy."""
    rows = [dict(n=3, l_seg=0.02, R=0.02, P=3000.0, obs=[(0, 0.05, 0.028, 0.01, 0.0)]),
            dict(n=4, l_seg=0.02, R=0.02, P=3000.0, obs=[(1, 0.07, -0.02, 0.01, 0.01), (0, 0.03, 0.03, 0.008, 0.0)],
                 acts=[(0.0, 2.0, 1, 5000.0, 0.02)]),
            dict(n=3, l_seg=0.02, R=0.025, P=5000.0, obs=[(1, 0.065, 0.0, 0.01, 0.03)])]
    sc = scene_of(rows)
    o = oracle.Oracle(sc, oracle.default_params(tol=1e-12))
    st = grow(o, 4)
    for i in range(3):
        th = o.theta_of(st, i)
        N = th.size
        x0 = np.concatenate([np.zeros(N), [0.0]])
        x0[:N - 1] = th[:N - 1]  # previous equilibrium with a fresh link, as the oracle starts
        st2 = o.new_state()
        o.run(st2, N - 1)
        x0[:N - 1] = o.theta_of(st2, i)
        lseg = float(sc["l_seg"][i])
        fun = lambda x: o.energy(i, x[:N], x[N], hessian=False)[0]
        jac = lambda x: o.energy(i, x[:N], x[N], hessian=False)[1]
        res = optimize.minimize(fun, x0, jac=jac, method="L-BFGS-B",
                                bounds=[(None, None)] * N + [(0.0, lseg)],
                                options=dict(ftol=1e-16, gtol=1e-13, maxiter=20000, maxcor=30))
        assert np.allclose(res.x[:N], th, atol=2e-6)
        assert res.x[N] == pytest.approx(st["l"][i], abs=2e-7)


# ------------------------------------------------------------------ P8 symmetry
def test_mirror_symmetry():
    sc = scenes.parity_batch(12)
    mir = {k: v.copy() for k, v in sc.items()}
    mir["obs_cy"] = -sc["obs_cy"]
    mir["act_side"] = -sc["act_side"]
    o1, o2 = oracle.Oracle(sc), oracle.Oracle(mir)
    s1, s2 = grow(o1, 20), grow(o2, 20)
    assert np.array_equal(s1["N"], s2["N"])
    assert np.allclose(s1["theta"], -s2["theta"], atol=1e-9)
    assert np.allclose(s1["l"], s2["l"], atol=1e-10)


def test_rigid_motion_equivariance():
    """Translating base and obstacles, or rotating both by 90 degrees (boxes swap
    half-sizes), leaves the joint angles unchanged."""
    sc = scenes.design_batch(6)
    sh = {k: v.copy() for k, v in sc.items()}
    for k, dv in (("obs_cx", 0.25), ("obs_cy", -0.5)):
        sh[k] = (sc[k].astype(np.float64) + dv).astype(np.float32)
    sh["base"] = sc["base"].copy()
    sh["base"][:, 0] += np.float32(0.25)
    sh["base"][:, 1] += np.float32(-0.5)
    rot = {k: v.copy() for k, v in sc.items()}
    rot["obs_cx"], rot["obs_cy"] = -sc["obs_cy"], sc["obs_cx"].copy()
    box = sc["obs_kind"] == 1
    rot["obs_a"] = np.where(box, sc["obs_b"], sc["obs_a"]).astype(np.float32)
    rot["obs_b"] = np.where(box, sc["obs_a"], sc["obs_b"]).astype(np.float32)
    rot["base"] = sc["base"].copy()
    rot["base"][:, 2] = np.float32(PI / 2)
    st = [grow(oracle.Oracle(s, oracle.default_params(tol=1e-10)), 25) for s in (sc, sh, rot)]
    # translation by float32-exact offsets changes only rounding
    assert np.allclose(st[0]["theta"], st[1]["theta"], atol=1e-7)
    assert np.allclose(st[0]["theta"], st[2]["theta"], atol=1e-7)


# ------------------------------------------------------------------ convergence test
def test_converged_state_close_to_tight_solve():
    """The state at tol 1e-6 (with its final step applied) is within 1e-4 link
    lengths of the state solved to 1e-12 from the same warm start."""
    sc = scenes.parity_batch(16)
    o6 = oracle.Oracle(sc)
    o12 = oracle.Oracle(sc, oracle.default_params(tol=1e-12))
    s = grow(o6, 19)
    for i in range(16):
        th = np.concatenate([o6.theta_of(s, i), [0.0]])
        a = o6.solve(i, th, 0.0)
        b = o12.solve(i, th, 0.0)
        assert a[4] == 0 and b[4] == 0
        pa, pb = o6.poses(i, a[0], a[1]), o12.poses(i, b[0], b[1])
        assert np.max(np.hypot(pa[0] - pb[0], pa[1] - pb[1])) < 1e-4 * 0.02
