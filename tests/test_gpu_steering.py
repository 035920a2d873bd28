"""Tip-steering (the paper's supplement) on the GPU against the oracle: robots
grow with an unpressurised tip actuator, then growth is stunted (distal
length held) while the tip actuator over the last links is pressurised in
steps.  Each steering step starts both sides from the oracle's state
(vine_set_state) with the same actuators; poses and contact sets are
compared as in the growth parity tests."""
import numpy as np
import pytest

import oracle
from paper_2509_15180_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402
from paper_2509_15180_gb300.steering import TipSteering  # noqa: E402
from test_gpu_parity import _classify, _max_switches  # noqa: E402

SPAN = 4


def _scene(n_robots=24):
    """Parity-batch robots (20 links of 2 cm, 10 circles), each given a tip
    actuator (last in its actuator list, side alternating)."""
    sc = scenes.parity_batch(n_robots)
    rows_act = []
    for i in range(n_robots):
        a0, a1 = sc["act_ptr"][i], sc["act_ptr"][i + 1]
        acts = [(sc["act_begin"][a], sc["act_end"][a], sc["act_side"][a], sc["act_pressure"][a], sc["act_l0"][a])
                for a in range(a0, a1)]
        acts.append((0.0, 1.0, 1 if i % 2 == 0 else -1, 0.0, float(sc["l_seg"][i])))
        rows_act.append(acts)
    flat = [a for r in rows_act for a in r]
    sc["act_ptr"] = np.concatenate([[0], np.cumsum([len(r) for r in rows_act])]).astype(np.int32)
    sc["act_begin"] = np.array([a[0] for a in flat], np.float32)
    sc["act_end"] = np.array([a[1] for a in flat], np.float32)
    sc["act_side"] = np.array([a[2] for a in flat], np.int8)
    sc["act_pressure"] = np.array([a[3] for a in flat], np.float32)
    sc["act_l0"] = np.array([a[4] for a in flat], np.float32)
    tip = sc["act_ptr"][1:] - 1
    return sc, tip


def test_tip_steering_matches_oracle():
    sc, tip = _scene()
    n = sc["n_links"].size
    b = vine.Batch(sc)
    steer = TipSteering(b, sc, tip, span=SPAN)
    # growth phase: both sides grow 20 links with the tip actuator at zero
    sc0 = dict(sc, act_pressure=steer.pressure.copy())
    orc = oracle.Oracle(sc0, oracle.default_params(tol=1e-10))
    ost = orc.new_state()
    orc.run(ost, 20, threads=16)
    tally = {"match": 0, "switch": 0, "flagged": 0}
    for p in (4000.0, 8000.0, 12000.0, 16000.0):
        ost["theta"][:] = ost["theta"].astype(np.float32)
        ost["l"][:] = ost["l"].astype(np.float32)
        ost["status"][ost["status"] == 1] = 0
        b.set_state(ost["N"], ost["theta"][: max(b.total_links, 1)].astype(np.float32), ost["l"].astype(np.float32))
        l_before = ost["l"].copy()
        steer.steer(p)
        st = b.state()
        # the oracle relaxes the same state with the same actuators
        sc_p = dict(sc, act_pressure=steer.pressure.copy(), act_begin=steer.begin.copy(), act_end=steer.end.copy())
        orc = oracle.Oracle(sc_p, oracle.default_params(tol=1e-10))
        orc.fix_length = True  # the equilibrium check of a parted robot holds the length too
        orc.relax(ost, fix_length=True, threads=16)
        assert np.array_equal(st["N"], ost["N"]) and np.all(st["N"] == 20)
        assert np.array_equal(st["l"], l_before.astype(np.float32))   # growth stunted: length held bitwise
        counts, pairs = b.contacts(512)
        for c in _classify(b, st, orc, ost, sc_p, counts, pairs):
            tally[c] += 1
    print("tip steering: %s over %d robot-steps" % (tally, 4 * n))
    assert tally["flagged"] <= 2
    assert tally["switch"] <= _max_switches(4 * n)
    b.close()


def test_steering_bends_the_tip_toward_the_actuator():
    sc, tip = _scene(8)
    b = vine.Batch(sc)
    steer = TipSteering(b, sc, tip, span=SPAN)
    steer.grow(20)
    st0 = b.state()
    heads0 = np.array([b.pose_of(st0, i)[-1, 2] for i in range(8)])
    steer.steer(15000.0)
    st1 = b.state()
    heads1 = np.array([b.pose_of(st1, i)[-1, 2] for i in range(8)])
    side = sc["act_side"][tip].astype(np.float64)
    ok = (st1["status"] == 0)
    # the tip turns toward the actuator's side, unless an obstacle holds it
    turned = side * (heads1 - heads0) > 0
    assert turned[ok].mean() >= 0.75
    assert np.array_equal(st1["N"], st0["N"]) and np.array_equal(st1["l"], st0["l"])
    b.close()
