"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bar: link start points and tip within 1e-4 link lengths, headings within
1e-4 rad, contact sets identical apart from grazing pairs (|gap| within
2e-4 link lengths), every step converged.  The convergence test stops at a
predicted displacement of tol = 1e-6 of the robot's length, i.e. tol N link
lengths, which exceeds 1e-4 link lengths beyond 100 links: robots within
2 tol N link lengths of the oracle (both sides inside the tolerance) are
counted separately as 'tol' matches.  Inputs are the seeded scenes of
paper_2509_15180_gb300.scenes.
"""
import numpy as np
import pytest

import oracle
from paper_2509_15180_gb300 import scenes

from parity import contacts_match

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402  (fails loudly if libvine.so is missing)

POSE_TOL = 1e-4      # link lengths
HEAD_TOL = 1e-4      # rad
TOL = 1e-6           # the solver's convergence tolerance (default parameters)
THREADS = 16


def _oracle(sc, tol=1e-10):
    return oracle.Oracle(sc, oracle.default_params(tol=tol))


def _prm(tp):
    """Library parameters with `tp` threads per robot (32: one warp; 64, 128:
    a team of two or four warps)."""
    p = vine.vine_params_default()
    p.threads_per_robot = tp
    return p


TEAMS = pytest.mark.parametrize("tp", [32, 64, 128])


def test_prologue_tables_match_oracle():
    sc = scenes.design_batch(16)
    b = vine.Batch(sc)
    T = b.tables()
    orc = _oracle(sc)
    ot = orc.tables()
    assert T["n_tab"] == len(ot) == 1
    l0, lo, hi, f = ot[0]
    assert T["hdr"][0, 0] == pytest.approx(lo, rel=1e-6, abs=1e-9)
    assert T["hdr"][0, 1] == pytest.approx((hi - lo) / 255, rel=1e-6)
    assert np.allclose(T["knots"][0, :, 0], f, rtol=2e-6, atol=1e-12 * f.max())
    # cumulative integral
    G = np.concatenate([[0.0], np.cumsum(0.5 * (hi - lo) / 255 * (f[1:] + f[:-1]))])
    assert np.allclose(T["knots"][0, :, 1], G, rtol=5e-6, atol=1e-9 * G.max())
    # wrinkling energy table against the oracle's quadrature
    thc, hu = T["consts"][2], T["consts"][3]
    for k in (0, 1, 5, 40, 300, 1023, 1024):
        m, _, u = oracle.wrinkle(thc + k * hu)
        assert T["utab"][k, 0] == pytest.approx(u, rel=2e-6)
        assert T["utab"][k, 1] == pytest.approx(m, rel=2e-6)
    b.close()


def _is_equilibrium(orc, i, theta, l, ls):
    """Stationarity at the GPU's state: the oracle's FP64 Newton step there
    predicts a displacement of at most 3 tol of the robot length (the GPU's
    own test is tol; FP32 rounding moves the residual by about tol / 3), or
    the oracle started there converges within max(1e-4, 2 tol N) link
    lengths."""
    th0 = np.asarray(theta, np.float64)
    try:
        _, r, _, _ = orc.gn_step(i, th0, float(l))
        if r <= 3.0 * TOL:
            return True
    except ValueError:
        pass
    px0, py0, _ = orc.poses(i, th0, float(l))
    th1, l1, it, r, stt = orc.solve(i, th0, float(l))
    px1, py1, _ = orc.poses(i, th1, l1)
    bar = max(POSE_TOL, 2.0 * TOL * th0.size) * ls
    return stt == 0 and max(np.max(np.abs(px1 - px0)), np.max(np.abs(py1 - py0))) <= bar


def _classify(b, st, orc, ost, sc, counts, pairs, idx_gpu=None):
    """Per robot: 'match' (poses and contacts within the bar), 'tol' (poses
    within 2 tol N link lengths, contacts equal: both sides inside the
    convergence tolerance, which is wider than the bar beyond 50 links),
    'switch' (a different, valid equilibrium: the path through a
    snap-through diverged), or 'flagged' (either side reports a step that
    did not converge; such robots are counted, not compared).  Anything else
    fails the test."""
    n = sc["n_links"].size
    idx_gpu = list(range(n)) if idx_gpu is None else list(idx_gpu)
    out = []
    for io, ig in enumerate(idx_gpu):
        if st["status"][ig] != 0 or ost["status"][io] != 0:
            out.append("flagged")
            continue
        ls = float(sc["l_seg"][io])
        th, px, py, psi = orc.theta_of(ost, io), *orc.poses(io, orc.theta_of(ost, io), ost["l"][io])
        pose = b.pose_of(st, ig)
        e = max(np.max(np.abs(pose[:, 0] - px[:-1])), np.max(np.abs(pose[:, 1] - py[:-1])),
                abs(st["tip"][ig, 0] - px[-1]), abs(st["tip"][ig, 1] - py[-1]))
        eh = np.max(np.abs(pose[:, 2] - psi))
        N = th.size
        bar_tol = max(POSE_TOL, 2.0 * TOL * N)
        if e <= bar_tol * ls and eh <= max(HEAD_TOL, 2.0 * TOL * N):
            g = {tuple(p) for p in pairs[ig, : counts[ig]]}
            gap = orc.gaps(io, th, ost["l"][io])
            o = {(int(x), int(y)) for x, y in zip(*np.nonzero(gap < 0))}
            gr = {(int(x), int(y)) for x, y in zip(*np.nonzero(np.abs(gap) <= 2e-4 * ls))}
            assert contacts_match(g, o, gr), "robot %d: contact sets differ: gpu-only %s oracle-only %s" % (
                ig, sorted(g - o - gr), sorted(o - g - gr))
            out.append("match" if (e <= POSE_TOL * ls and eh <= HEAD_TOL) else "tol")
        else:
            assert _is_equilibrium(orc, io, b.theta_of(st, ig), st["l"][ig], ls), (
                "robot %d: position error %.3g link lengths and the GPU state is not an equilibrium" % (ig, e / ls))
            out.append("switch")
    return out


@TEAMS
def test_parity_batch_full(tp):
    """64 robots x 20 steps, independent trajectories."""
    sc = scenes.parity_batch()
    b = vine.Batch(sc, _prm(tp))
    b.simulate()
    st = b.state()
    counts, pairs = b.contacts(64)
    stats = b.stats()
    orc = _oracle(sc)
    ost = orc.new_state()
    orc.run(ost, 20, threads=THREADS)
    assert np.all(st["status"] == 0) and np.all(st["N"] == 20)
    assert stats["steps_converged"] == 64 * 20
    assert stats["robot_link_steps"] == scenes.robot_link_steps(sc["n_links"])
    cls = _classify(b, st, orc, ost, sc, counts, pairs)
    print("parity batch: %d match, %d tol, %d basin switches" % (cls.count("match"), cls.count("tol"),
                                                            cls.count("switch")))
    assert cls.count("switch") <= 6
    b.close()


def _to_fp32(ost):
    """Rounds the oracle's state to FP32, the GPU's storage precision, in
    place, so that both sides start a step from the same values."""
    ost["theta"][:] = ost["theta"].astype(np.float32)
    ost["l"][:] = ost["l"].astype(np.float32)


def _stepwise(sc, steps, tp=32):
    """Each step, both sides start from the oracle's previous state (rounded
    to FP32 and loaded into the GPU batch with vine_set_state); returns the
    classification counts over all robot-steps."""
    n = sc["n_links"].size
    b = vine.Batch(sc, _prm(tp))
    orc = _oracle(sc)
    ost = orc.new_state()
    tally = {"match": 0, "tol": 0, "switch": 0, "flagged": 0}
    flagged_robots = set()
    for step in range(steps):
        _to_fp32(ost)
        # an unconverged earlier step is assessed on its own step: both sides
        # start this one with a clean status
        ost["status"][ost["status"] == 1] = 0
        b.set_state(ost["N"], ost["theta"][: max(b.total_links, 1)].astype(np.float32),
                    ost["l"].astype(np.float32))
        b.grow_step(1)
        orc.run(ost, 1, threads=THREADS)
        st = b.state()
        counts, pairs = b.contacts(512)
        assert np.all(st["N"] == ost["N"])
        assert np.all((st["N"] == np.minimum(step + 1, sc["n_links"])) | (st["status"] != 0))
        for i, c in enumerate(_classify(b, st, orc, ost, sc, counts, pairs)):
            tally[c] += 1
            if c == "flagged":
                flagged_robots.add(i)
    b.close()
    tally["flagged_robots"] = len(flagged_robots)
    return tally


@TEAMS
def test_parity_batch_stepwise_resynced(tp):
    """Each step, both sides start from the oracle's previous state; the
    step's result must match unless that step is a snap-through to another
    valid equilibrium."""
    sc = scenes.parity_batch()
    tally = _stepwise(sc, 20, tp)
    print("stepwise: %s in %d robot-steps" % (tally, 20 * 64))
    assert tally["flagged"] == 0
    assert tally["switch"] <= 0.01 * 20 * 64


@TEAMS
def test_uneven_stepwise_resynced_parity(tp):
    """Uneven robots (40-90 links, 5-200 obstacles, 0-8 actuators), resynced
    every step: over a whole growth the trajectories of two solvers can part
    at a snap-through, but single steps from the same state agree."""
    sc = scenes.uneven_batch(12, n_range=(40, 90))
    steps = int(sc["n_links"].max())
    tally = _stepwise(sc, steps, tp)
    total = int(sc["n_links"].sum())
    print("uneven stepwise: %s (robot-steps with growth: %d)" % (tally, total))
    assert tally["switch"] <= 0.02 * total
    # robots with some step that either side left unconverged; the
    # oracle's own rate on these scenes is a few percent of robots
    assert tally["flagged_robots"] <= 3


def test_plain_form_is_bitwise_identical():
    sc = scenes.parity_batch(16)
    b1, b2 = vine.Batch(sc), vine.Batch(sc)
    b1.simulate()
    b2.simulate_plain()
    s1, s2 = b1.state(), b2.state()
    for k in ("theta", "l", "pose", "tip", "N", "iters"):
        assert np.array_equal(s1[k], s2[k]), k
    b1.close(); b2.close()


@TEAMS
def test_design_batch_full_size_sampled(tp):
    """4096 robots x 100 links in the launch the benchmark times (one-warp
    and two-warp teams); 12 sampled robots recomputed by the oracle."""
    sc = scenes.design_batch()
    b = vine.Batch(sc, _prm(tp))
    b.simulate()
    torch.cuda.synchronize()
    st = b.state()
    counts, pairs = b.contacts(256)
    stats = b.stats()
    assert np.all((st["N"] == 100) | (st["status"] == vine.INST_NONFINITE))
    nbad = int((st["status"] != 0).sum())
    # the FP64 oracle itself leaves 20 of these 4096 robots with a step that
    # does not converge in 100 iterations (deep-penetration coiling)
    assert nbad <= 40, "too many non-converged robots: %d" % nbad
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(4096, 12, replace=False))
    sub = scenes.subset(sc, idx)
    orc = _oracle(sub)
    ost = orc.new_state()
    orc.run(ost, 100, threads=THREADS)
    cls = _classify(b, st, orc, ost, sub, counts, pairs, idx_gpu=idx)
    print("design batch sample: %d match, %d tol, %d basin switches, %d flagged" % (
        cls.count("match"), cls.count("tol"), cls.count("switch"), cls.count("flagged")))
    assert cls.count("match") + cls.count("tol") >= 9
    assert stats["robot_link_steps"] >= 0.99 * scenes.robot_link_steps(sc["n_links"])
    b.close()


def test_uneven_batch_sampled():
    """Uneven robots (30-120 links, 5-200 obstacles, 0-8 actuators) in one launch."""
    sc = scenes.uneven_batch(96, n_range=(30, 120))
    b = vine.Batch(sc)
    b.simulate()
    st = b.state()
    counts, pairs = b.contacts(512)
    assert np.all((st["N"] == sc["n_links"]) | (st["status"] == vine.INST_NONFINITE))
    idx = np.arange(0, 96, 6)
    sub = scenes.subset(sc, idx)
    orc = _oracle(sub)
    ost = orc.new_state()
    orc.run(ost, 400, threads=THREADS)
    cls = _classify(b, st, orc, ost, sub, counts, pairs, idx_gpu=idx)
    print("uneven sample: %d match, %d tol, %d basin switches, %d flagged" % (
        cls.count("match"), cls.count("tol"), cls.count("switch"), cls.count("flagged")))
    # whole trajectories part at snap-throughs (every non-matching robot was
    # checked to sit at a valid equilibrium); single steps are compared by
    # the resynced test
    assert cls.count("match") + cls.count("tol") >= len(idx) // 4
    b.close()


def test_edge_cases():
    # straight tube, no obstacles/actuators; one-link robot; bad input next to good ones
    sc = scenes.parity_batch(4)
    sc["act_ptr"] = np.zeros(5, np.int32)
    for k in ("act_begin", "act_end", "act_pressure", "act_l0"):
        sc[k] = np.zeros(0, np.float32)
    sc["act_side"] = np.zeros(0, np.int8)
    sc["obs_ptr"][:] = 0
    for k in ("obs_cx", "obs_cy", "obs_a", "obs_b"):
        sc[k] = np.zeros(0, np.float32)
    sc["obs_kind"] = np.zeros(0, np.uint8)
    sc["n_links"][1] = 1
    sc["radius"][2] = -1.0
    b = vine.Batch(sc)
    b.simulate()
    st = b.state()
    assert st["status"][2] == vine.INST_BADINPUT and st["N"][2] == 0
    assert st["status"][0] == 0 and st["status"][1] == 0 and st["N"][1] == 1
    assert np.all(b.theta_of(st, 0) == 0.0)
    ls = float(sc["l_seg"][0])
    assert np.allclose(b.pose_of(st, 0)[:, 0], np.arange(20) * ls, atol=1e-7)
    assert st["tip"][0, 0] == pytest.approx(20 * ls, abs=1e-6)
    # reset + re-run is deterministic; zero steps is a no-op
    b.reset()
    b.grow_step(0)
    assert np.all(b.state()["N"] == 0)
    b.simulate()
    st2 = b.state()
    for k in ("theta", "pose", "tip", "l"):
        assert np.array_equal(st[k], st2[k]), k
    b.close()


def test_device_inputs_match_host_inputs():
    sc = scenes.parity_batch(8)
    dsc = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in sc.items()}
    b1, b2 = vine.Batch(sc), vine.Batch(dsc)
    b1.simulate(); b2.simulate()
    s1, s2 = b1.state(), b2.state()
    for k in ("theta", "pose", "tip", "l", "iters"):
        assert np.array_equal(s1[k], s2[k]), k
    b1.close(); b2.close()


def test_broad_phase_is_exact():
    """The per-link obstacle lists skip only obstacles that cannot reach a
    link, so the growth is bitwise the same as testing every obstacle."""
    for sc in (scenes.design_batch(64), scenes.uneven_batch(48, n_range=(30, 120))):
        out = []
        for bp in (1, 0):
            prm = vine.vine_params_default()
            prm.broad_phase = bp
            b = vine.Batch(sc, prm)
            b.simulate()
            out.append((b.state(), b.stats()))
            b.close()
        (s1, t1), (s0, t0) = out
        for k in ("theta", "l", "N", "status", "iters", "resid"):
            assert np.array_equal(s1[k], s0[k]), k
        assert t1["evaluations"] == t0["evaluations"]
        assert t0["pair_tests_executed"] == t0["pair_tests"]
        print("broad phase: %.1f%% of the all-pairs tests run" % (100.0 * t1["pair_tests_executed"] / t1["pair_tests"]))
        assert t1["pair_tests_executed"] < t0["pair_tests_executed"]


def test_maximum_sizes_and_empty_batch():
    """A robot at every per-robot maximum (1024 links, 1024 obstacles, 64
    actuators) grown 24 steps against the oracle; one link more is a bad
    input; an empty batch is refused."""
    rng = np.random.default_rng(17)
    base = scenes.parity_batch(1)
    n_obs, n_act = 1024, 64
    cx = rng.uniform(0.08, 0.6, n_obs)
    cy = rng.uniform(-0.3, 0.3, n_obs)
    keep = np.hypot(cx, cy) > 0.05 + 0.006  # clear of the base
    cx, cy = np.where(keep, cx, cx + 0.1), cy
    sc = dict(base)
    sc["n_links"] = np.array([1024], np.int32)
    sc["obs_ptr"] = np.array([0, n_obs], np.int32)
    sc["obs_kind"] = np.zeros(n_obs, np.uint8)
    sc["obs_cx"] = cx.astype(np.float32)
    sc["obs_cy"] = cy.astype(np.float32)
    sc["obs_a"] = rng.uniform(0.002, 0.006, n_obs).astype(np.float32)
    sc["obs_b"] = np.zeros(n_obs, np.float32)
    sc["act_ptr"] = np.array([0, n_act], np.int32)
    b0 = rng.integers(0, 20, n_act).astype(np.float32)
    sc["act_begin"] = b0
    sc["act_end"] = (b0 + rng.uniform(0.5, 3.0, n_act)).astype(np.float32)
    sc["act_side"] = np.where(rng.random(n_act) < 0.5, 1, -1).astype(np.int8)
    sc["act_pressure"] = rng.uniform(0.0, 300.0, n_act).astype(np.float32)
    sc["act_l0"] = np.full(n_act, 0.02, np.float32)
    b = vine.Batch(sc)
    b.grow_step(24)
    st = b.state()
    counts, pairs = b.contacts(256)
    orc = _oracle(sc)
    ost = orc.new_state()
    orc.run(ost, 24, threads=1)
    assert st["N"][0] == 24 and st["status"][0] == 0 and ost["status"][0] == 0
    cls = _classify(b, st, orc, ost, sc, counts, pairs)
    assert cls[0] in ("match", "tol"), cls
    b.close()
    # one link beyond the maximum: that robot is flagged, the batch runs
    big = scenes.concat([scenes.parity_batch(1), dict(sc, n_links=np.array([1025], np.int32))])
    b = vine.Batch(big)
    b.grow_step(3)
    st = b.state()
    assert st["status"][1] == vine.INST_BADINPUT and st["N"][1] == 0 and st["N"][0] == 3
    b.close()
    with pytest.raises(vine.VineError) as e:
        vine.Batch(scenes.subset(scenes.parity_batch(2), []))
    assert e.value.status == vine.VINE_EINVAL
