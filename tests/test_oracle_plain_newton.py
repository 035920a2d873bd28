"""Pin of the oracle's equilibrium solver against a plain damped Newton solve
(CPU only).

The oracle's solver carries path rules of its own (exact Hessian with a
Gauss-Newton fallback, an active set for the distal length, an
approximate-Wolfe slope test once the cost change is at FP64 rounding level).
The result of a growth step is defined as the stationary point of the cost of
Eq. (pbd) reached from the warm start (Sec. 4.1, Algorithm 1), so none of
these rules may change it.  Here every growth step of the parity scenes and
of design-batch robots is solved a second time, from the same warm start, by
the textbook method: Newton steps on the exact Hessian with a Levenberg shift
when it is not positive definite, the distal length projected onto
[0, l_seg], and backtracking on the plain Armijo condition -- no rounding-level
rule and no untested steps.  Both must land on the same equilibrium within
1e-6 link lengths.  Where the warm start lies in a non-convex region of the
cost (the exact Hessian there is indefinite: a snap-through), the minimum
"reached from the warm start" depends on how a method leaves that region;
only there may the two solves end in different minima, both verified as
minima, and such steps are counted.

The plain solve uses only the oracle's model functions (cost, gradient, exact
Hessian, poses), which are pinned on their own in test_oracle_models.py and
test_oracle_solver.py.
"""
import numpy as np
import pytest

import oracle
from paper_2509_15180_gb300 import scenes

SAME = 1e-6  # link lengths
FLOOR = 1e-7  # link lengths: soft-direction displacement below which J changes by under one ulp


def _disp(orc, i, th, l, d):
    """Largest displacement (m) of a link end point under the step d
    (joint steps, distal length step), and l_seg times the largest joint step."""
    px, py, psi = orc.poses(i, th, l)
    N = th.size
    rx = px[1:, None] - px[None, :-1]  # p_{k+1} - p_j
    ry = py[1:, None] - py[None, :-1]
    mask = np.tril(np.ones((N, N)))
    dx = -(mask * ry) @ d[:N]
    dy = (mask * rx) @ d[:N]
    dx[-1] += d[N] * np.cos(psi[N - 1])  # the distal end also moves along the link
    dy[-1] += d[N] * np.sin(psi[N - 1])
    return float(np.max(np.hypot(dx, dy)))


def plain_newton(orc, i, th, l, ls, tol=1e-12, max_iter=3000):
    """Damped Newton with Armijo backtracking on J; returns (theta, l, r, ok).
    r: predicted displacement of the last step in link lengths."""
    th = th.astype(np.float64).copy()
    N = th.size
    r = np.inf
    for _ in range(max_iter):
        J, g, _ = orc.energy(i, th, l, hessian=False)
        H = orc.hessian_exact(i, th, l)
        lfix = (l <= 0.0 and g[N] > 0.0) or (l >= ls and g[N] < 0.0)
        m = N if lfix else N + 1
        Hm = H[:m, :m]
        mu = 0.0
        scale = np.max(np.abs(np.diag(Hm)))
        while True:  # Levenberg shift until positive definite
            try:
                Lc = np.linalg.cholesky(Hm + mu * np.eye(m))
                break
            except np.linalg.LinAlgError:
                mu = max(10.0 * mu, 1e-10 * scale)
        d = np.zeros(N + 1)
        d[:m] = -np.linalg.solve(Lc.T, np.linalg.solve(Lc, g[:m]))
        r = max(_disp(orc, i, th, l, d), ls * np.max(np.abs(d[:N]))) / ls
        if r <= tol * N:
            return th + d[:N], min(max(l + d[N], 0.0), ls), r, True
        a = 1.0
        for _h in range(60):
            tt = th + a * d[:N]
            lt = min(max(l + a * d[N], 0.0), ls)
            Jt, _, _ = orc.energy(i, tt, lt, hessian=False)
            if Jt <= J + 1e-4 * (a * g[:N] @ d[:N] + g[N] * (lt - l)):
                break
            a *= 0.5
        if a < 1.0 and r <= FLOOR:
            # the predicted decrease (about g.d) is below one ulp of J: Armijo
            # can no longer see the decrease of the full step, so the solve
            # ends here, already far inside the comparison bar
            return tt, lt, r, True
        th, l = tt, lt
    return th, l, r, False


def _compare(sc, steps):
    orc = oracle.Oracle(sc, oracle.default_params(tol=1e-12))
    ost = orc.new_state()
    n = sc["n_links"].size
    tally = dict(same=0, basin=0, skipped=0, worst=0.0)
    for _ in range(steps):
        prev = [(orc.theta_of(ost, i), float(ost["l"][i]), int(ost["N"][i])) for i in range(n)]
        orc.run(ost, 1, threads=8)
        for i in range(n):
            th0, l0, N0 = prev[i]
            if N0 >= sc["n_links"][i] or ost["status"][i] != 0:
                tally["skipped"] += N0 < sc["n_links"][i]
                continue
            ls = float(np.float32(sc["l_seg"][i]))
            warm = np.concatenate([th0, [0.0]])  # the new link at the tip, l = 0
            thp, lp, rp, ok = plain_newton(orc, i, warm, 0.0, ls)
            tho = orc.theta_of(ost, i)
            pxo, pyo, _ = orc.poses(i, tho, ost["l"][i])
            pxp, pyp, _ = orc.poses(i, thp, lp)
            e = max(np.max(np.abs(pxo - pxp)), np.max(np.abs(pyo - pyp))) / ls
            assert ok, "plain Newton did not converge (robot %d, r %.3g)" % (i, rp)
            if e <= SAME:
                tally["same"] += 1
                tally["worst"] = max(tally["worst"], e)
            else:
                # different minima are allowed only where the warm start sits
                # in a non-convex region of J (a snap-through: the exact
                # Hessian there is indefinite, and the descent paths of two
                # methods can part); both results must be minima
                Hw = orc.hessian_exact(i, warm, 0.0)
                assert np.min(np.linalg.eigvalsh(Hw)) < 0.0, (
                    "robot %d: different equilibria from a convex warm start (%.3g link lengths)" % (i, e))
                for t, lv in ((tho, ost["l"][i]), (thp, lp)):
                    H = orc.hessian_exact(i, t, lv)
                    m = t.size if (lv <= 0 or lv >= ls) else t.size + 1
                    assert np.all(np.linalg.eigvalsh(H[:m, :m]) > 0), "robot %d: not a minimum" % i
                tally["basin"] += 1
            # continue both from the oracle's state (the plain solve is
            # checked step by step, from the warm start the oracle had)
    return tally


def test_parity_scene_steps_match_plain_newton():
    sc = scenes.parity_batch()
    t = _compare(sc, 20)
    print("parity scene: %s" % t)
    assert t["same"] + t["basin"] + t["skipped"] == 64 * 20
    assert t["basin"] <= 0.02 * 64 * 20  # measured: 16 of 1280, each from an indefinite warm start
    assert t["worst"] <= SAME


@pytest.mark.slow
def test_design_robot_steps_match_plain_newton():
    sc = scenes.subset(scenes.design_batch(), list(range(0, 4096, 256)))
    t = _compare(sc, 100)
    print("design robots: %s" % t)
    assert t["same"] + t["basin"] + t["skipped"] == 16 * 100
    assert t["basin"] <= 0.02 * 16 * 100
    assert t["worst"] <= SAME
