"""Pins for the oracle's component models (CPU only).

Each test ties the oracle to something other than itself: SciPy's elliptic
integrals and quadrature, Gauss's arithmetic-geometric mean, closed forms
of the paper's equations, or series expansions derived by hand.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize, special

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def test_defaults_match_paper_constants():
    g = json.load(open(GOLD))
    P = oracle.default_params()
    assert P.a_spam == g["a_spam"]
    assert (P.w_a, P.w_b, P.w_c) == (g["w_a"], g["w_b"], g["w_c"])
    assert P.R_c == g["R_c_m"] and P.R_act == g["R_act_m"]


# ---------------------------------------------------------------- elliptic
@pytest.mark.parametrize("m", [0.0, 1e-6, 0.01, 0.1, 0.3, 0.5, 0.7, 0.9])
def test_elliptic_vs_scipy(m):
    for phi in np.linspace(0.0, math.pi / 2, 23):
        assert oracle.ellip_F(phi, m) == pytest.approx(special.ellipkinc(phi, m), rel=1e-13, abs=1e-15)
        assert oracle.ellip_E(phi, m) == pytest.approx(special.ellipeinc(phi, m), rel=1e-13, abs=1e-15)


def _agm_KE(m):
    """Complete integrals from Gauss's AGM: K = pi / (2 AGM(1, sqrt(1-m))),
    E = K (1 - sum 2^(n-1) c_n^2)."""
    a, b, c = 1.0, math.sqrt(1.0 - m), math.sqrt(m)
    s, p2 = 0.5 * c * c, 0.5
    for _ in range(40):
        a, b, c = 0.5 * (a + b), math.sqrt(a * b), 0.5 * (a - b)
        p2 *= 2.0
        s += p2 * c * c
    K = math.pi / (2.0 * a)
    return K, K * (1.0 - s)


@pytest.mark.parametrize("m", [0.05, 0.25, 0.5, 0.8])
def test_complete_integrals_vs_agm(m):
    K, E = _agm_KE(m)
    assert oracle.ellip_F(math.pi / 2, m) == pytest.approx(K, rel=1e-14)
    assert oracle.ellip_E(math.pi / 2, m) == pytest.approx(E, rel=1e-14)


def test_elliptic_m0_is_phi():
    for phi in (0.1, 0.7, 1.3):
        assert oracle.ellip_F(phi, 0.0) == pytest.approx(phi, rel=1e-15)
        assert oracle.ellip_E(phi, 0.0) == pytest.approx(phi, rel=1e-15)


# ---------------------------------------------------------------- sPAM model
RC, RACT, A = 0.005, 0.01718, 1e-4
PHI_SAT = math.acos(RC / RACT)


def _sp_eq2(phi, m, la, a=A):
    c = math.cos(phi)
    return special.ellipkinc(phi, m) / (math.sqrt(m) * c) - (la / RC) * (1 + a / (2 * m * c * c))


def _sp_eq1(phi, m, la, l0, eps):
    c = math.cos(phi)
    lhs = (special.ellipeinc(phi, m) - 0.5 * special.ellipkinc(phi, m)) / (math.sqrt(m) * c)
    return lhs - la / (2 * RC) * (1 - l0 / la * eps)


@pytest.mark.parametrize("l0", [0.01, 0.015, 0.02, 0.03, 0.05, 0.08])
def test_spam_solution_satisfies_equations(l0):
    """Eq. (sPAM_1), (sPAM_2), (phiRC), (sPAM_force) hold at the oracle's solution,
    evaluated with SciPy's elliptic integrals."""
    for m in (0.002, 0.01, 0.05, 0.1, 0.2, 0.3, 0.4, 0.49, 0.5):
        eps, f, phi, sat = oracle.spam_eval(m, l0)
        if sat:
            assert phi == pytest.approx(PHI_SAT, rel=1e-15)
            c = math.cos(phi)
            la = RC * special.ellipkinc(phi, m) / (math.sqrt(m) * c) / (1 + A / (2 * m * c * c))
            assert _sp_eq2(phi, m, la) == pytest.approx(0.0, abs=1e-9 * l0 / RC)
        else:
            la = l0
            assert phi <= PHI_SAT
            assert _sp_eq2(phi, m, la) == pytest.approx(0.0, abs=1e-9 * l0 / RC)
        assert _sp_eq1(phi, m, la, l0, eps) == pytest.approx(0.0, abs=1e-9 * l0 / RC)
        c = math.cos(phi)
        assert f == pytest.approx(math.pi * RC ** 2 * (1 - 2 * m) / (2 * m * c * c), rel=1e-14, abs=1e-20)


@pytest.mark.parametrize("l0", [0.01, 0.02, 0.03])
def test_spam_takes_smallest_root(l0):
    """No sign change of the Eq. (sPAM_2) residual below the chosen root; the
    second root lies beyond phi_sat (next to pi/2)."""
    for m in (0.01, 0.1, 0.3, 0.5):
        eps, f, phi, sat = oracle.spam_eval(m, l0)
        if sat:
            continue
        grid = np.linspace(1e-6, phi * (1 - 1e-9), 400)
        assert all(_sp_eq2(p, m, l0) < 0 for p in grid)
        # the other root
        hi = np.linspace(PHI_SAT, math.pi / 2 - 1e-9, 4000)
        vals = np.array([_sp_eq2(p, m, l0) for p in hi])
        assert (vals[:-1] * vals[1:] <= 0).sum() == 1
        k = int(np.nonzero(vals[:-1] * vals[1:] <= 0)[0][0])
        assert hi[k] > 1.5


def test_spam_force_vanishes_at_half():
    for l0 in (0.01, 0.02, 0.05):
        assert oracle.spam_eval(0.5, l0)[1] == 0.0


def test_spam_a0_reduces_to_ppam():
    """With a = 0 the unsaturated branch solves the ideal PPAM relation
    F(phi, m) / (sqrt(m) cos phi) = l_0 / R_c."""
    P = oracle.default_params(a_spam=0.0)
    for m in (0.05, 0.2, 0.4):
        eps, f, phi, sat = oracle.spam_eval(m, 0.02, P)
        assert not sat
        assert _sp_eq2(phi, m, 0.02, a=0.0) == pytest.approx(0.0, abs=1e-9)


def test_spam_saturation_continuous():
    """The branch switch at phi = phi_sat is continuous in eps and f (l0 = 5 cm
    saturates for large m)."""
    l0 = 0.05
    ms = np.linspace(0.05, 0.5, 400)
    sats = [oracle.spam_eval(m, l0)[3] for m in ms]
    assert any(sats) and not all(sats)
    k = sats.index(True)
    lo, hi = ms[k - 1], ms[k]
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if oracle.spam_eval(mid, l0)[3]:
            hi = mid
        else:
            lo = mid
    e0, f0 = oracle.spam_eval(lo, l0)[:2]
    e1, f1 = oracle.spam_eval(hi, l0)[:2]
    assert abs(e1 - e0) < 1e-7 and abs(f1 - f0) < 1e-7 * abs(f0)


@pytest.mark.parametrize("l0", [0.01, 0.015, 0.02, 0.025, 0.03])
def test_spam_monotone(l0):
    """eps increases and F_t decreases with m on the tabulated range, so the
    strain table is single valued and force falls with contraction."""
    ms = np.linspace(0.002, 0.5, 300)
    ev = np.array([oracle.spam_eval(m, l0)[:2] for m in ms])
    assert np.all(np.diff(ev[:, 0]) > 0)
    assert np.all(np.diff(ev[:, 1]) < 0)


def test_spam_table_knots():
    l0 = 0.015
    lo, hi, f = oracle.spam_table(l0)
    assert lo == pytest.approx(oracle.spam_eval(0.002, l0)[0], rel=1e-15)
    assert hi == pytest.approx(oracle.spam_eval(0.5, l0)[0], rel=1e-15)
    assert f[0] == pytest.approx(oracle.spam_eval(0.002, l0)[1], rel=1e-15)
    assert f[-1] == 0.0
    assert np.all(np.diff(f) < 0)
    h = (hi - lo) / (oracle.NKNOT - 1)
    for k in (1, 17, 64, 128, 200, 254):
        target = lo + k * h
        m = optimize.brentq(lambda mm: oracle.spam_eval(mm, l0)[0] - target, 0.002, 0.5, xtol=1e-15, rtol=1e-15)
        assert f[k] == pytest.approx(oracle.spam_eval(m, l0)[1], rel=1e-9)


def test_table_interpolant():
    lo, hi, f = oracle.spam_table(0.02)
    fv = lambda e: oracle.table_eval(lo, hi, f, e)[0]
    # held below, zero above
    assert fv(lo - 0.1) == f[0] and oracle.table_eval(lo, hi, f, lo - 0.1)[1] == 0.0
    assert fv(hi + 0.1) == 0.0
    # integral from 0 against SciPy quadrature of the interpolant
    h = (hi - lo) / (oracle.NKNOT - 1)
    knots = list(lo + h * np.arange(oracle.NKNOT))
    for e in (-0.05, -0.01, 0.0, 0.013, 0.2, hi + 0.05):
        pts = [k for k in knots if min(0.0, e) < k < max(0.0, e)]
        ref = integrate.quad(fv, 0.0, e, points=pts or None, limit=800, epsabs=1e-16, epsrel=1e-13)[0]
        assert oracle.table_eval(lo, hi, f, e)[2] == pytest.approx(ref, rel=1e-9, abs=1e-16)
    # slope is the finite difference inside a cell
    e = lo + 10.3 * h
    d = 1e-3 * h
    assert oracle.table_eval(lo, hi, f, e)[1] == pytest.approx((fv(e + d) - fv(e - d)) / (2 * d), rel=1e-7)


# ---------------------------------------------------------------- wrinkling moment
EC = 0.01
THC = 2 * math.asin(EC)


def _mhat_asin(th, ec=EC):
    """Same moment written through gamma_0 = 2 asin(sqrt(1 - eps_c / s))."""
    a = abs(th)
    s = math.sin(min(a, math.pi) / 2)
    g = 2 * math.asin(math.sqrt(1 - ec / s))
    v = (math.sin(2 * g) + 2 * math.pi - 2 * g) / (4 * (math.sin(g) + (math.pi - g) * math.cos(g)))
    return math.copysign(v, th)


def test_wrinkle_onset_value():
    """At onset gamma_0 = 0 and Eq. (wrinkling_model) gives M = pi P R^3 / 2."""
    assert oracle.wrinkle(THC)[0] == pytest.approx(0.5, rel=1e-15)
    assert oracle.wrinkle(THC * (1 + 1e-12))[0] == pytest.approx(0.5, rel=1e-9)


def test_wrinkle_acos_equals_asin_form():
    for th in np.concatenate([np.linspace(THC * 1.0001, math.pi, 200), [3.5, -0.3, -2.0]]):
        assert oracle.wrinkle(th)[0] == pytest.approx(_mhat_asin(th), rel=1e-12)


def test_wrinkle_series_near_onset():
    """M/(pi P R^3) = 1/2 + g^2/4 - g^3/(2 pi) + O(g^4) for small gamma_0."""
    for s_rel in (1e-6, 1e-5, 1e-4):
        s = EC * (1 + s_rel)
        th = 2 * math.asin(s)
        g = math.acos(2 * EC / s - 1)
        assert oracle.wrinkle(th)[0] == pytest.approx(0.5 + g * g / 4 - g ** 3 / (2 * math.pi), abs=5 * g ** 4)


def test_wrinkle_full_limit():
    """As eps_c -> 0 the moment at theta = pi tends to the fully wrinkled pi P R^3."""
    assert oracle.wrinkle(math.pi, 1e-8)[0] == pytest.approx(1.0, abs=2e-4)


def test_wrinkle_monotone_odd_ramp():
    ths = np.linspace(0, math.pi, 2000)
    m = np.array([oracle.wrinkle(t, energy=False)[0] for t in ths])
    assert np.all(np.diff(m) > 0)
    for t in (0.001, 0.01, 0.5, 2.0):
        assert oracle.wrinkle(-t)[0] == -oracle.wrinkle(t)[0]
    for t in (0.0, 0.3 * THC, THC):
        assert oracle.wrinkle(t)[0] == pytest.approx(t / (2 * THC), rel=1e-15, abs=0)


def test_wrinkle_derivative_fd():
    for th in (0.2 * THC, THC * 1.5, 0.1, 0.7, 2.5, 3.1, -0.4):
        h = 1e-5 * min(1.0, abs(th))
        fd = (oracle.wrinkle(th + h)[0] - oracle.wrinkle(th - h)[0]) / (2 * h)
        assert oracle.wrinkle(th)[1] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_wrinkle_energy_vs_quad():
    for th in (0.5 * THC, THC, 0.05, 0.5, 2.0, 3.0, 3.3, -1.0):
        ref = integrate.quad(lambda t: oracle.wrinkle(t, energy=False)[0], 0.0, th, points=[THC] if abs(th) > THC else None,
                             limit=400, epsabs=1e-14, epsrel=1e-12)[0]
        assert oracle.wrinkle(th)[2] == pytest.approx(ref, rel=1e-10, abs=1e-14)
    assert oracle.wrinkle(0.5 * THC)[2] == pytest.approx((0.5 * THC) ** 2 / (4 * THC), rel=1e-15)
