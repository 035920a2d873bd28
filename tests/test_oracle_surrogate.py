"""Pins of the surrogate oracle (oracle/surrogate.py, Sec. 4.3): the loss
gradient against central differences, the ReLU network against a loop over
units written out, Adam's first step against its closed form, and the
training data against the exact sPAM model (phi on the saturated branch,
the force formula)."""
import math

import numpy as np
import pytest

import oracle
from oracle import surrogate as sg


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    th = sg.he_init(rng) + 0.05 * rng.standard_normal(sg.N_PARAM)
    x = rng.uniform(0, 1, (40, 2))
    t = rng.uniform(0, 1, (40, 2))
    _, g = sg.loss_and_grad(th, x, t)
    h = 1e-6
    for k in rng.choice(sg.N_PARAM, 40, replace=False):
        e = np.zeros(sg.N_PARAM)
        e[k] = h
        fd = (sg.loss_and_grad(th + e, x, t)[0] - sg.loss_and_grad(th - e, x, t)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9), k


def test_forward_against_unit_loops():
    rng = np.random.default_rng(1)
    th = sg.he_init(rng) + 0.1 * rng.standard_normal(sg.N_PARAM)
    x = rng.uniform(-1, 1, (5, 2))
    W1, b1, W2, b2 = sg.unpack(th)
    y = sg.forward(th, x)
    for s in range(5):
        for k in range(2):
            acc = b2[k]
            for j in range(sg.H):
                a = b1[j] + W1[j, 0] * x[s, 0] + W1[j, 1] * x[s, 1]
                acc += W2[k, j] * max(a, 0.0)
            assert y[s, k] == pytest.approx(acc, rel=1e-14, abs=1e-14)


def test_adam_first_step_closed_form():
    # after one step from zero moments the bias-corrected step is lr * sign(g)
    th = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    new, m, v = sg.adam(th, g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(new, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_data_is_the_sPAM_model():
    p = oracle.default_params()
    phi_sat = math.acos(p.R_c / p.R_act)
    for m, l0 in ((0.01, 0.02), (0.2, 0.05), (0.45, 0.08), (0.002, 0.03)):
        eps, f, phi, sat = oracle.spam_eval(m, l0, p)
        assert 0.0 < phi <= phi_sat + 1e-12
        if sat:
            assert phi == pytest.approx(phi_sat, rel=1e-12)
        # Eq. sPAM_force per unit pressure
        assert f == pytest.approx(math.pi * p.R_c ** 2 * (1 - 2 * m) / (2 * m * math.cos(phi) ** 2), rel=1e-12)
