"""Oracle for the actuator design synthesis of Sec. 4.2.

TEST INFRASTRUCTURE ONLY: the tests are the only users; the product package
never imports this module.  Written from the definitions, one pair at a
time, with SciPy's brentq as the scalar root finder and the FP64 oracle
(vine_oracle.c, through ``oracle``) for the model functions.

Reading of Sec. 4.2 (the paper parameterises an actuator by the turning
angle it produces and inverts the sPAM model for pressure and cell length,
picking the highest pressure among the feasible designs on discrete sets):
* a design (P, l0) holds a free joint (no contact) of the body at the angle
  theta_eq(P, l0) > 0 where the wrinkling moment balances the actuator
  moment (Eq. wrinkling_model against Eq. sPAM_force times the moment arm
  2 R + R_act, Sec. 3.3), with the actuator strain d theta / l_seg and the
  force per pressure taken from the cell length's sPAM table (the same
  piecewise-linear table on 256 strain knots the growth step uses; zero
  force beyond the table's strain range, its first knot below it);
  theta_eq = pi when the actuator still wins at pi;
* a design is feasible for a target theta_t when |theta_eq - theta_t| <= tol;
* among the feasible designs: the highest pressure, then the closest angle,
  then the shorter cell (the paper favours pressure over cell length);
  none feasible: index -1.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import optimize

import oracle


def joint_equilibrium(P: float, l0: float, R: float, Pv: float, ls: float, params=None, table=None) -> float:
    """theta_eq(P, l0): the root in (0, pi] of the free-joint balance.
    table: (eps_lo, eps_hi, f) of the cell length, if already built."""
    prm = params or oracle.default_params()
    d = 2.0 * R + prm.R_act
    lo, hi, fk = table if table is not None else oracle.spam_table(l0, prm)
    M0 = math.pi * Pv * R ** 3

    def h(th):
        m = oracle.wrinkle(th, prm.eps_crit, energy=False)[0]
        f = oracle.table_eval(lo, hi, fk, d * th / ls)[0]
        return M0 * m - P * f * d

    if h(math.pi) <= 0.0:
        return math.pi
    if h(0.0) >= 0.0:
        return 0.0
    return optimize.brentq(h, 0.0, math.pi, xtol=1e-15, rtol=1e-15, maxiter=500)


def pair_table(pressures, l0_grid, R, Pv, ls, params=None) -> np.ndarray:
    """theta_eq for every (pressure, cell length): [n_p, n_l0]."""
    tabs = [oracle.spam_table(float(l0), params or oracle.default_params()) for l0 in l0_grid]
    return np.array([[joint_equilibrium(float(P), float(l0), R, Pv, ls, params, tabs[k])
                      for k, l0 in enumerate(l0_grid)] for P in pressures])


def choose(theta_t: float, pairs: np.ndarray, pressures, tol: float):
    """(p_index, l0_index) by the selection rule, (-1, -1) when none is feasible."""
    best = None
    for ip, P in enumerate(pressures):
        for il in range(pairs.shape[1]):
            dev = abs(pairs[ip, il] - theta_t)
            if dev > tol:
                continue
            key = (-float(P), dev, il, ip)
            if best is None or key < best[0]:
                best = (key, ip, il)
    return (-1, -1) if best is None else (best[1], best[2])


def synthesize(theta_targets, pressures, l0_grid, R, Pv, ls, tol, params=None):
    """Per target: (p_index, l0_index, theta_eq of the choice or NaN); and the pair table."""
    pairs = pair_table(pressures, l0_grid, R, Pv, ls, params)
    out = []
    for t in theta_targets:
        ip, il = choose(float(t), pairs, pressures, tol)
        out.append((ip, il, pairs[ip, il] if ip >= 0 else float("nan")))
    return out, pairs
