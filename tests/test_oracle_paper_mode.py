"""Pins of the oracle's literal Algorithm 1 mode (mode 1: actuator force
frozen at the step's initial strain, fixed-rate gradient descent)."""
import numpy as np

import oracle
from paper_2509_15180_gb300 import scenes


def _bare(n_inst, n_links):
    sc = scenes.parity_batch(n_inst)
    sc["n_links"] = np.full(n_inst, n_links, np.int32)
    sc["act_ptr"] = np.zeros(n_inst + 1, np.int32)
    for k in ("act_begin", "act_end", "act_pressure", "act_l0"):
        sc[k] = np.zeros(0, np.float32)
    sc["act_side"] = np.zeros(0, np.int8)
    sc["obs_ptr"] = np.zeros(n_inst + 1, np.int32)
    for k in ("obs_cx", "obs_cy", "obs_a", "obs_b"):
        sc[k] = np.zeros(0, np.float32)
    sc["obs_kind"] = np.zeros(0, np.uint8)
    return sc


def test_growth_follows_the_geometric_closed_form():
    """No actuators, no obstacles: each step the distal length moves a
    fraction gd_alpha of the way to l_seg (the growth spring is quadratic)
    and the chain stays straight."""
    sc = _bare(2, 5)
    for alpha, K in ((0.05, 50), (0.3, 7)):
        P = oracle.default_params(mode=1, gd_alpha=alpha, gd_steps=K)
        orc = oracle.Oracle(sc, P)
        st = orc.new_state()
        orc.run(st, 3, threads=1)
        ls = float(sc["l_seg"][0])
        assert np.allclose(st["l"], ls * (1.0 - (1.0 - alpha) ** K), rtol=1e-13, atol=0)
        assert np.all(orc.theta_of(st, 0) == 0.0) and np.all(st["N"] == 3)


def test_one_actuated_joint_below_onset_follows_the_linear_recursion():
    """One link under an actuator, below wrinkling onset: the frozen force
    gives a constant moment tau = s P_a f(0) d, the joint sees the ramp
    stiffness w_a pi P R^3 / (2 theta_c), so theta_K = theta* (1 - (1 -
    alpha)^K) with theta* = 2 theta_c tau / (pi P R^3)."""
    sc = _bare(1, 1)
    sc["act_ptr"] = np.array([0, 1], np.int32)
    sc["act_begin"] = np.array([0.0], np.float32)
    sc["act_end"] = np.array([1.0], np.float32)
    sc["act_side"] = np.array([1], np.int8)
    sc["act_pressure"] = np.array([5.0], np.float32)  # small: stays below onset
    sc["act_l0"] = np.array([0.02], np.float32)
    alpha, K = 0.2, 9
    P = oracle.default_params(mode=1, gd_alpha=alpha, gd_steps=K)
    orc = oracle.Oracle(sc, P)
    st = orc.new_state()
    orc.run(st, 1, threads=1)
    l0, lo, hi, f = orc.tables()[0]
    f0, _, _ = oracle.table_eval(lo, hi, f, 0.0)
    R, Pv = float(sc["radius"][0]), float(sc["pressure"][0])
    d = 2.0 * R + P.R_act
    tau = 5.0 * f0 * d
    thc = 2.0 * np.arcsin(P.eps_crit)
    theta_star = 2.0 * thc * tau / (np.pi * Pv * R ** 3)
    assert 0.0 < theta_star < thc
    want = theta_star * (1.0 - (1.0 - alpha) ** K)
    got = orc.theta_of(st, 0)[0]
    assert abs(got - want) <= 1e-12 * theta_star


def test_one_descent_step_is_the_preconditioned_gradient_step():
    """Without actuators the frozen-force cost is the equilibrium mode's cost:
    one step of mode 1 from a grown state equals x - alpha grad J(x) with the
    step sizes gd_alpha 2 theta_c / (w_a pi P R^3) (joint angles) and
    gd_alpha / (2 w_b k_g) (distal length), using the gradient of the
    separately pinned cost (the new link starts at theta = 0, l = 0)."""
    sc = scenes.parity_batch(6)
    sc["act_ptr"] = np.zeros(7, np.int32)
    for k in ("act_begin", "act_end", "act_pressure", "act_l0"):
        sc[k] = np.zeros(0, np.float32)
    sc["act_side"] = np.zeros(0, np.int8)
    nt = oracle.Oracle(sc, oracle.default_params(tol=1e-12))
    st = nt.new_state()
    nt.run(st, 12, threads=6)  # a grown state with contacts
    alpha = 0.03
    P = oracle.default_params(mode=1, gd_alpha=alpha, gd_steps=1)
    gd = oracle.Oracle(sc, P)
    s1 = {k: v.copy() for k, v in st.items()}
    gd.run(s1, 1, threads=1)
    thc = 2.0 * np.arcsin(P.eps_crit)
    for i in range(6):
        th0 = np.concatenate([nt.theta_of(st, i), [0.0]])
        _, g, _ = nt.energy(i, th0, 0.0, hessian=False)
        R, Pv, ls = float(sc["radius"][i]), float(sc["pressure"][i]), float(sc["l_seg"][i])
        a_th = alpha * 2.0 * thc / (P.w_a * np.pi * Pv * R ** 3)
        kg = np.pi * Pv * R ** 2 / (2.0 * ls)
        a_l = alpha / (2.0 * P.w_b * kg)
        want_th = th0 - a_th * g[:-1]
        want_l = min(max(0.0 - a_l * g[-1], 0.0), ls)
        assert np.allclose(gd.theta_of(s1, i), want_th, rtol=1e-13, atol=1e-16)
        assert abs(s1["l"][i] - want_l) <= 1e-15 * ls
