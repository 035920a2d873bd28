"""Pins of the oracle's relaxation at the present links (tip-steering of
the paper's supplement): a relaxation at an equilibrium stays there, the
held distal length does not move, and a tip actuator on a straight chain in
free space bends exactly its joints to the decoupled scalar balance."""
import numpy as np
import pytest

import oracle
from test_oracle_solver import _free_joint_balance, scene_of


def _rows(p_tip, n=10, k=4, extra=()):
    return [dict(n=n, l_seg=0.02, R=0.025, P=5000.0, acts=list(extra) + [(float(n - k), float(n), 1, p_tip, 0.02)])]


def test_relax_at_equilibrium_stays():
    sc = scene_of(_rows(0.0, extra=[(1.0, 5.0, -1, 8000.0, 0.02)]) +
                  [dict(n=12, l_seg=0.015, R=0.03, P=4000.0, acts=[(0.0, 6.0, 1, 9000.0, 0.015)],
                        obs=[(0, 0.12, 0.05, 0.03, 0.0)])])
    o = oracle.Oracle(sc, oracle.default_params(tol=1e-12))
    st = o.new_state()
    o.run(st, 12)
    th0, l0 = st["theta"].copy(), st["l"].copy()
    it0 = st["iters"].copy()
    for fix in (True, False):
        o.relax(st, fix_length=fix)
        assert np.all(st["status"] == 0)
        assert np.allclose(st["theta"], th0, atol=1e-9, rtol=0)
        assert np.allclose(st["l"], l0, atol=1e-12, rtol=0)
    # a state already at equilibrium needs at most one Newton step per relaxation
    assert np.all(st["iters"] - it0 <= 2 * 2)


def test_tip_actuator_on_straight_chain_is_the_scalar_balance():
    n, k, p_tip = 10, 4, 12000.0
    o0 = oracle.Oracle(scene_of(_rows(0.0, n, k)), oracle.default_params(tol=1e-12))
    st = o0.new_state()
    o0.run(st, n)
    assert np.all(o0.theta_of(st, 0) == 0.0)
    l_before = float(st["l"][0])
    sc = scene_of(_rows(p_tip, n, k))
    o = oracle.Oracle(sc, oracle.default_params(tol=1e-12))
    o.relax(st, fix_length=True)
    th = o.theta_of(st, 0)
    assert st["status"][0] == 0 and st["N"][0] == n
    assert float(st["l"][0]) == l_before          # growth stunted: the length is held exactly
    assert np.all(th[: n - k] == 0.0)              # uncovered joints carry no moment
    for j in range(n - k, n):
        assert th[j] == pytest.approx(_free_joint_balance(o, sc, 0, j, -1.0, 1.0), abs=1e-10)
    assert np.all(th[n - k:] > 0)                  # side +1 bends toward positive angles


def test_tip_heading_grows_with_pressure():
    n, k = 12, 5
    o0 = oracle.Oracle(scene_of(_rows(0.0, n, k)), oracle.default_params(tol=1e-12))
    st0 = o0.new_state()
    o0.run(st0, n)
    heads = []
    for p in (2000.0, 6000.0, 12000.0, 20000.0):
        st = {kk: v.copy() for kk, v in st0.items()}
        o = oracle.Oracle(scene_of(_rows(p, n, k)), oracle.default_params(tol=1e-12))
        o.relax(st, fix_length=True)
        heads.append(o.theta_of(st, 0).sum())
    assert np.all(np.diff(heads) > 0) and heads[0] > 0
