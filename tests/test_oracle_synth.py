"""Pins of the design-synthesis oracle (Sec. 4.2, oracle/synth.py): the
scalar joint equilibrium against the oracle's full chain solver, its
monotonicity, the selection rule on a hand-made table, and a synthesised
design reproducing its target in the oracle's growth simulation."""
import math

import numpy as np
import pytest

import oracle
from oracle import synth
from test_oracle_solver import scene_of

R, PV, LS = 0.03335, 10342.0, 0.025


def _grow_one(P, l0, n=6, tol=1e-12):
    sc = scene_of([dict(n=n, l_seg=LS, R=R, P=PV, acts=[(0.0, float(n), 1, P, l0)])])
    o = oracle.Oracle(sc, oracle.default_params(tol=tol))
    st = o.new_state()
    o.run(st, n)
    assert st["status"][0] == 0
    return o.theta_of(st, 0)


@pytest.mark.parametrize("P,l0", [(20000.0, 0.025), (60000.0, 0.031), (5000.0, 0.02)])
def test_joint_equilibrium_equals_the_chain_solver(P, l0):
    f32 = lambda v: float(np.float32(v))  # the scene stores float32 inputs
    th = _grow_one(P, l0)
    ref = synth.joint_equilibrium(f32(P), f32(l0), f32(R), f32(PV), f32(LS))
    assert np.allclose(th, ref, atol=1e-9, rtol=0), (th, ref)


def test_equilibrium_grows_with_pressure():
    th = [synth.joint_equilibrium(P, 0.025, R, PV, LS) for P in (5e3, 1e4, 2e4, 4e4, 8e4)]
    assert all(b > a for a, b in zip(th, th[1:])) and th[0] > 0


def test_selection_rule_on_a_hand_made_table():
    pressures = [10.0, 20.0, 30.0]
    pairs = np.array([[0.50, 0.52, 0.40],
                      [0.49, 0.505, 0.70],
                      [0.80, 0.90, 1.00]])
    # target 0.5, tol 0.02: P=30 none; P=20: l0 0 (0.01 off) and l0 1 (0.005 off): the closer
    assert synth.choose(0.5, pairs, pressures, 0.02) == (1, 1)
    # equal deviation at the highest feasible pressure: the shorter cell
    pairs2 = np.array([[0.5, 0.5, 0.5], [0.51, 0.49, 0.7], [0.8, 0.9, 1.0]])
    assert synth.choose(0.5, pairs2, pressures, 0.02) == (1, 0)
    assert synth.choose(0.1, pairs, pressures, 0.02) == (-1, -1)
    assert synth.choose(1.0, pairs, pressures, 0.0) == (2, 2)


def test_synthesised_design_reproduces_its_target():
    pressures = np.arange(10e3, 100e3 + 1, 10e3)
    grid = 0.020 + 0.001 * np.arange(0, 61, 6)   # coarse grid keeps the pin quick
    targets = [0.03, 0.06, 0.09]   # per-joint angles this body reaches (up to about 0.1 rad)
    out, pairs = synth.synthesize(targets, pressures, grid, R, PV, LS, tol=0.01)
    assert np.all(np.diff(pairs, axis=0) > 0)   # every cell length: angle grows with pressure
    for t, (ip, il, th_eq) in zip(targets, out):
        assert ip >= 0, t
        # no feasible design at a higher pressure
        assert not np.any(np.abs(pairs[ip + 1:] - t) <= 0.01)
        th = _grow_one(float(pressures[ip]), float(grid[il]), tol=1e-10)
        assert np.all(np.abs(th - t) <= 0.01 + 1e-6), (t, th)
