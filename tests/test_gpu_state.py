"""vine_set_state: growth continued from a loaded state (the warm start of
Algorithm 2's propagation from stored tree nodes) is bitwise the growth
continued in place; invalid states mark only their robot."""
import numpy as np
import pytest

from paper_2509_15180_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402

GEOM = ("theta", "l", "N", "tip", "pose")
KEYS = GEOM + ("status",)


def test_continue_from_loaded_state_is_bitwise_in_place():
    sc = scenes.uneven_batch(48, n_range=(20, 60))
    a = vine.Batch(sc)
    a.grow_step(12)
    mid = a.state()
    a.simulate()
    end_a = a.state()
    b = vine.Batch(sc)
    b.set_state(mid["N"], mid["theta"], mid["l"])
    st = b.state()
    for k in GEOM:
        assert np.array_equal(st[k], mid[k]), k
    # the state is loaded with the validation status: a step that ran out of
    # iterations before the state was taken is not carried
    assert np.all(st["status"] == 0) and np.all(st["iters"] == 0)
    b.simulate()
    end_b = b.state()
    # robots whose step failed before the state was taken stopped there in
    # the first batch; loaded with a clean status, they grow on in the second
    clean = mid["status"] == 0
    for i in np.nonzero(clean)[0]:
        for k in ("theta", "pose"):
            assert np.array_equal(a.theta_of(end_a, i) if k == "theta" else a.pose_of(end_a, i),
                                  b.theta_of(end_b, i) if k == "theta" else b.pose_of(end_b, i)), (k, i)
    for k in ("l", "N", "tip", "status", "iters"):
        x = end_a[k][clean] - (mid[k][clean] if k == "iters" else 0)  # counters restart at the loaded state
        assert np.array_equal(x, end_b[k][clean]), k
    for i in np.nonzero(~clean)[0]:
        assert end_a["N"][i] == mid["N"][i] and end_b["N"][i] >= mid["N"][i]
    a.close()
    b.close()


def test_device_state_equals_host_state():
    sc = scenes.parity_batch(16)
    a = vine.Batch(sc)
    a.grow_step(7)
    mid = a.state()
    b1, b2 = vine.Batch(sc), vine.Batch(sc)
    b1.set_state(mid["N"], mid["theta"], mid["l"])
    dev = torch.device("cuda")
    b2.set_state(torch.from_numpy(mid["N"]).to(dev), torch.from_numpy(mid["theta"]).to(dev),
                 torch.from_numpy(mid["l"]).to(dev))
    torch.cuda.synchronize()
    b1.simulate()
    b2.simulate()
    s1, s2 = b1.state(), b2.state()
    for k in KEYS:
        assert np.array_equal(s1[k], s2[k]), k
    for x in (a, b1, b2):
        x.close()


def test_invalid_state_marks_only_its_robot():
    sc = scenes.parity_batch(8)
    b = vine.Batch(sc)
    b.grow_step(5)
    st = b.state()
    N, th, l = st["N"].copy(), st["theta"].copy(), st["l"].copy()
    N[1] = int(sc["n_links"][1]) + 1                     # more links than the target
    th[b.offsets[2] + 1] = np.nan                        # non-finite angle
    l[3] = float(sc["l_seg"][3]) * 1.5                   # distal length beyond l_seg
    l[4] = -1e-3                                         # negative distal length
    N[5] = 0                                             # empty robot: its angles are ignored
    th[b.offsets[5]: b.offsets[5] + 5] = np.nan
    b.set_state(N, th, l)
    s = b.state()
    for i in (1, 2, 3, 4):
        assert s["status"][i] == vine.INST_BADINPUT and s["N"][i] == 0, i
    for i in (0, 5, 6, 7):
        assert s["status"][i] == 0, i
    assert s["N"][5] == 0 and np.all(b.theta_of(s, 5) == 0)
    b.simulate()
    s = b.state()
    assert np.all(s["N"][[0, 5, 6, 7]] == sc["n_links"][[0, 5, 6, 7]])
    assert np.all(s["N"][[1, 2, 3, 4]] == 0)
    # a valid state clears the mark
    b.set_state(st["N"], st["theta"], st["l"])
    assert np.all(b.state()["status"] == 0)
    b.close()
