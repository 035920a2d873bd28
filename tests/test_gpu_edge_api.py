"""Edge cases of the entry points added for the planner, tip-steering, design
synthesis and the surrogate: empty inputs, robots without links or with bad
input, mode 1, unreachable targets."""
import numpy as np
import pytest

from paper_2509_15180_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import surrogate, vine  # noqa: E402


def test_relax_skips_empty_and_bad_robots():
    sc = scenes.parity_batch(6)
    b = vine.Batch(sc)
    b.grow_step(8)
    st = b.state()
    N, th, l = st["N"].copy(), st["theta"].copy(), st["l"].copy()
    N[1] = 0                      # no links: nothing to relax
    l[2] = -1.0                   # bad state: BADINPUT, left empty
    b.set_state(N, th, l)
    b.relax(fix_length=True)
    s = b.state()
    assert s["N"][1] == 0 and s["status"][1] == 0 and np.all(b.theta_of(s, 1) == 0)
    assert s["status"][2] == vine.INST_BADINPUT and s["N"][2] == 0
    for i in (0, 3, 4, 5):
        assert s["N"][i] == 8 and s["l"][i] == l[i]
    assert b.stats()["steps_total"] == 4      # one relaxation per robot with links
    with pytest.raises(vine.VineError):
        vine._check(vine._lib.vine_relax(b.h, 2, None), "vine_relax")
    b.close()


def test_mode1_relax_holds_length_and_counts_descent_steps():
    sc = scenes.parity_batch(8)
    p = vine.vine_params_default()
    p.mode = 1
    b = vine.Batch(sc, p)
    b.grow_step(6)
    st = b.state()
    b.set_state(st["N"], st["theta"], st["l"])
    b.relax(fix_length=True)
    s = b.state()
    assert np.array_equal(s["N"], st["N"]) and np.array_equal(s["l"], st["l"])
    assert np.all(s["iters"] == p.gd_steps)
    b.close()


def test_empty_calls():
    g = vine.synthesize([], 0.03335, 10342.0, 0.025, [1e4], 0.02, 0.001, 3, 0.01)
    assert g["p_index"].size == 0 and g["pairs"].shape == (1, 3)
    assert vine.sst_select(np.zeros((3, 3), np.float32), np.zeros(3), np.ones(3, np.uint8),
                           np.zeros((0, 3), np.float32), 1.0, 1.0).size == 0
    keep, deact = vine.sst_prune(np.zeros((0, 3), np.float32), np.zeros(0), np.zeros(0, np.uint8),
                                 np.zeros((0, 3), np.float32), np.zeros(0), 1.0, 1.0)
    assert keep.size == 0 and deact.size == 0
    x, y, _ = surrogate.make_dataset(64, 3)
    net = surrogate.init_net(x, 3)
    assert vine.surrogate_eval(net, np.zeros((0, 2))).shape == (0, 2)
    s = vine.spam_samples(np.zeros(0), np.zeros(0))
    assert s["eps"].size == 0


def test_unreachable_targets_and_invalid_samples():
    g = vine.synthesize([0.5, 3.0, -0.1], 0.03335, 10342.0, 0.025, [1e4, 2e4], 0.02, 0.001, 61, 0.004)
    assert np.all(g["p_index"] == -1) and np.all(g["l0_index"] == -1) and np.all(np.isnan(g["theta_eq"]))
    with pytest.raises(vine.VineError):
        vine.spam_samples([0.6], [0.02])          # m beyond 1/2
    with pytest.raises(vine.VineError):
        vine.spam_samples([0.1], [-0.02])         # negative cell length
    x, y, _ = surrogate.make_dataset(64, 4)
    net = surrogate.init_net(x, 4)
    bad = dict(net, in_scale=np.zeros(2, np.float32))
    with pytest.raises(vine.VineError):
        vine.surrogate_eval(bad, x)
