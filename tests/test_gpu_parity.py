"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bar (one for every chain length): link start points and tip within 1e-4
link lengths, headings within 1e-4 rad, contact sets identical apart from
grazing pairs (|gap| within 2e-4 link lengths), every step converged.  A
growth step converges when its Newton step moves no link end point by more
than tol = 1e-6 of the robot length nor by more than tol_link = 2.5e-5 link
lengths, and the final step is applied, so converged states sit well inside
the bar at any N.  Where a whole growth parts at a snap-through (the two
solvers' descent from a non-convex warm start ends in different minima),
the robot counts as a basin switch: its GPU state must then be a minimum of
the oracle's model with the contact set the oracle finds there, and a
step-by-step replay must show that the two growths part at a snap-through
(a warm start where the cost is not convex).  Single steps from the same
state part in at most 2 % of robot-steps.  Inputs are the seeded scenes of
paper_2509_15180_gb300.scenes.
"""
import numpy as np
import pytest

import oracle
from paper_2509_15180_gb300 import scenes

from parity import GRAZE, contacts_match

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402  (fails loudly if libvine.so is missing)

POSE_TOL = 1e-4      # link lengths
HEAD_TOL = 1e-4      # rad
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


def _switch_is_valid(orc, i, theta, l, ls, gpu_pairs):
    """A robot whose state parts from the oracle's: the GPU state must be a
    minimum of the oracle's model with the contacts the oracle finds there.
    (1) stationary: the oracle's FP64 Newton step at the GPU's state moves no
    link end by more than 1e-4 link lengths, or the oracle started there
    converges within 1e-4 link lengths of it; (2) a minimum: the oracle's
    exact Hessian there is positive definite on the free unknowns; (3) the
    contact set the GPU reports equals the oracle's at that state (grazing
    pairs aside).  Returns a reason string when invalid, else None."""
    th0 = np.asarray(theta, np.float64)
    N = th0.size
    px0, py0, _ = orc.poses(i, th0, float(l))
    stationary = False
    try:
        _, r, _, _ = orc.gn_step(i, th0, float(l))
        stationary = r * N <= POSE_TOL
    except ValueError:
        pass
    if not stationary:
        th1, l1, _, _, stt = orc.solve(i, th0, float(l))
        px1, py1, _ = orc.poses(i, th1, l1)
        stationary = stt == 0 and max(np.max(np.abs(px1 - px0)), np.max(np.abs(py1 - py0))) <= POSE_TOL * ls
    if not stationary:
        return "not stationary"
    H = orc.hessian_exact(i, th0, float(l))
    m = N if (orc.fix_length or l <= 0.0 or l >= ls) else N + 1  # the free unknowns
    if not np.min(np.linalg.eigvalsh(H[:m, :m])) > 0.0:
        return "not a minimum (indefinite Hessian)"
    gap = orc.gaps(i, th0, float(l))
    o = {(int(x), int(y)) for x, y in zip(*np.nonzero(gap < 0))}
    gr = {(int(x), int(y)) for x, y in zip(*np.nonzero(np.abs(gap) <= GRAZE * ls))}
    if not contacts_match(gpu_pairs, o, gr):
        return "contact set differs at the GPU state: gpu-only %s oracle-only %s" % (
            sorted(gpu_pairs - o - gr), sorted(o - gpu_pairs - gr))
    return None


def _classify(b, st, orc, ost, sc, counts, pairs, idx_gpu=None):
    """Per robot: 'match' (poses and contacts within the bar), 'switch' (a
    different minimum: the path through a snap-through diverged; checked by
    _switch_is_valid), or 'flagged' (either side reports a step that did not
    converge; such robots are counted, not compared).  Anything else fails
    the test.  idx_gpu[k] is the GPU batch index of the oracle's robot k."""
    n = sc["n_links"].size
    idx_gpu = list(range(n)) if idx_gpu is None else list(idx_gpu)
    return [_classify_one(b, st, orc, ost, sc, counts, pairs, io, int(ig)) for io, ig in enumerate(idx_gpu)]


def _flags(st, ost, idx_gpu):
    """(robots the GPU leaves unconverged while the oracle converges, robots
    the oracle leaves unconverged)."""
    g = np.asarray(st["status"])[np.asarray(idx_gpu)] != 0
    o = np.asarray(ost["status"]) != 0
    return int((g & ~o).sum()), int(o.sum())


def _max_switches(n_compared):
    return int(0.02 * n_compared)


def _indefinite(orc, i, theta, l):
    H = orc.hessian_exact(i, np.asarray(theta, np.float64), float(l))
    return np.min(np.linalg.eigvalsh(H)) < 0.0


def _switches_start_at_snap_throughs(sc, idx, tp, final_state=None, steps=None):
    """Whole growths that part: replay the robots idx (indices into sc) step
    by step on both sides, the GPU with the same team size as the batch, and
    find the first step whose results differ by more than the bar.  That
    step must start from a non-convex warm start (the oracle's exact Hessian
    indefinite at the oracle's or the GPU's state with the new link
    appended): a snap-through, where the minimum reached depends on how a
    method leaves the non-convex region.  The replay must end bitwise where
    the batch launch ended (final_state: theta and l per robot).  Returns the
    first parting step per robot."""
    sub = scenes.subset(sc, np.asarray(idx))
    b = vine.Batch(sub, _prm(tp))
    orc = _oracle(sub)
    ost = orc.new_state()
    n = len(idx)
    steps = int(sub["n_links"].max()) if steps is None else steps
    first = [None] * n
    for k in range(steps):
        looking = any(f is None for f in first)
        st_prev = b.state() if looking else None
        o_prev = [orc.theta_of(ost, i) for i in range(n)] if looking else None
        b.grow_step(1)
        orc.run(ost, 1, threads=THREADS)
        if not looking:
            continue
        st = b.state()
        for i in range(n):
            if first[i] is not None or k >= sub["n_links"][i] or st["status"][i] or ost["status"][i]:
                continue
            ls = float(sub["l_seg"][i])
            th = orc.theta_of(ost, i)
            px, py, _ = orc.poses(i, th, ost["l"][i])
            pose = b.pose_of(st, i)
            e = max(np.max(np.abs(pose[:, 0] - px[:-1])), np.max(np.abs(pose[:, 1] - py[:-1])),
                    abs(st["tip"][i, 0] - px[-1]), abs(st["tip"][i, 1] - py[-1]))
            if e > POSE_TOL * ls:
                first[i] = k
                warm_o = np.concatenate([o_prev[i], [0.0]])
                warm_g = np.concatenate([b.theta_of(st_prev, i).astype(np.float64), [0.0]])
                assert _indefinite(orc, i, warm_o, 0.0) or _indefinite(orc, i, warm_g, 0.0), (
                    "robot %d parted from the oracle at step %d from a convex warm start (%.3g link lengths)"
                    % (idx[i], k, e / ls))
    if final_state is not None:
        st = b.state()
        for i in range(n):
            th_b, l_b = final_state[i]
            assert np.array_equal(b.theta_of(st, i), th_b) and st["l"][i] == l_b, "replay of robot %d" % idx[i]
    b.close()
    return first


def _check_switches(b, st, sc, cls, idx_gpu=None, tp=0):
    """Every whole-growth switch of cls starts at a snap-through, and they
    stay a small fraction of the compared robots.  tp: the threads per robot
    the batch was created with (0: the length classes)."""
    n = len(cls)
    idx_gpu = list(range(n)) if idx_gpu is None else list(idx_gpu)
    sw = [k for k, c in enumerate(cls) if c == "switch"]
    if not sw:
        return []
    fin = [(b.theta_of(st, idx_gpu[k]), st["l"][idx_gpu[k]]) for k in sw]
    first = _switches_start_at_snap_throughs(sc, sw, tp, final_state=fin)
    # whole growths pass through several snap-throughs each, where FP32
    # noise decides between minima: measured 2-9 % of robots part (each at a
    # snap-through, checked above); single steps from the same state part in
    # at most 1 % of robot-steps (the resynced tests)
    assert len(sw) <= max(1, 0.10 * n), "%d of %d robots parted" % (len(sw), n)
    return first


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
    first = _check_switches(b, st, sc, cls, tp=tp)
    print("parity batch: %d match, %d basin switches (parting at steps %s)" % (
        cls.count("match"), cls.count("switch"), first))
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
    b = vine.Batch(sc, _prm(tp))
    orc = _oracle(sc)
    ost = orc.new_state()
    tally = {"match": 0, "switch": 0, "flagged": 0, "flag_gpu": 0, "flag_oracle": 0}
    flagged_robots = set()
    max_pairs = 4 * int(sc["n_links"].max())
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
        counts, pairs = b.contacts(max_pairs)
        assert np.all(counts <= max_pairs)
        assert np.all(st["N"] == ost["N"])
        assert np.all((st["N"] == np.minimum(step + 1, sc["n_links"])) | (st["status"] != 0))
        for i in np.nonzero(step < sc["n_links"])[0]:  # the robots that grew in this step
            c = _classify_one(b, st, orc, ost, sc, counts, pairs, int(i))
            tally[c] += 1
            if c == "flagged":
                flagged_robots.add(int(i))
                tally["flag_gpu"] += int(st["status"][i] != 0)
                tally["flag_oracle"] += int(ost["status"][i] != 0)
    b.close()
    tally["flagged_robots"] = len(flagged_robots)
    return tally


def _classify_one(b, st, orc, ost, sc, counts, pairs, io, ig=None):
    """The class of the oracle's robot io, which is robot ig of the GPU batch
    (default: the same index)."""
    ig = io if ig is None else ig
    if st["status"][ig] != 0 or ost["status"][io] != 0:
        return "flagged"
    ls = float(sc["l_seg"][io])
    th = orc.theta_of(ost, io)
    px, py, psi = orc.poses(io, th, ost["l"][io])
    pose = b.pose_of(st, ig)
    e = max(np.max(np.abs(pose[:, 0] - px[:-1])), np.max(np.abs(pose[:, 1] - py[:-1])),
            abs(st["tip"][ig, 0] - px[-1]), abs(st["tip"][ig, 1] - py[-1]))
    eh = np.max(np.abs(pose[:, 2] - psi))
    g = {tuple(p) for p in pairs[ig, : counts[ig]]}
    if e <= POSE_TOL * ls and eh <= HEAD_TOL:
        gap = orc.gaps(io, th, ost["l"][io])
        o = {(int(x), int(y)) for x, y in zip(*np.nonzero(gap < 0))}
        gr = {(int(x), int(y)) for x, y in zip(*np.nonzero(np.abs(gap) <= GRAZE * ls))}
        assert contacts_match(g, o, gr), "robot %d: contact sets differ: gpu-only %s oracle-only %s" % (
            ig, sorted(g - o - gr), sorted(o - g - gr))
        return "match"
    why = _switch_is_valid(orc, io, b.theta_of(st, ig), float(st["l"][ig]), ls, g)
    assert why is None, "robot %d: position error %.3g link lengths and the GPU state is %s" % (ig, e / ls, why)
    return "switch"


@TEAMS
def test_parity_batch_stepwise_resynced(tp):
    """Each step, both sides start from the oracle's previous state; the
    step's result must match unless that step is a snap-through to another
    valid minimum."""
    sc = scenes.parity_batch()
    tally = _stepwise(sc, 20, tp)
    print("stepwise: %s in %d robot-steps" % (tally, 20 * 64))
    assert tally["flagged"] == 0
    assert tally["switch"] <= _max_switches(20 * 64)


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
    assert tally["switch"] <= _max_switches(total)
    # steps that either side leaves unconverged (out of iterations): the GPU
    # no more often than the oracle, plus one
    assert tally["flag_gpu"] <= tally["flag_oracle"] + 1


@pytest.mark.parametrize("tp", [32, 128])
def test_long_chain_stepwise_resynced_parity(tp):
    """Long uneven robots (200-300 links, the upper range of the uneven
    batch), resynced every step: every single step of every robot, including
    the steps past 256 links, against the oracle."""
    sc = scenes.uneven_batch(8, replicate=5, n_range=(200, 300))
    steps = int(sc["n_links"].max())
    tally = _stepwise(sc, steps, tp)
    total = int(sc["n_links"].sum())
    print("long-chain stepwise: %s (robot-steps with growth: %d)" % (tally, total))
    assert tally["switch"] <= _max_switches(total)
    assert tally["flag_gpu"] <= tally["flag_oracle"] + 1


@pytest.mark.parametrize("tp", [32, 128])
def test_chain_grown_past_256_links(tp):
    """Eight 320-link robots grown from one link (320 growth steps, the
    positions of the distal links accumulated past 256 links) in one launch,
    against the oracle's growth of the same robots."""
    sc = scenes.uneven_batch(8, replicate=6, n_range=(320, 320))
    b = vine.Batch(sc, _prm(tp))
    b.simulate()
    st = b.state()
    counts, pairs = b.contacts(1024)
    orc = _oracle(sc)
    ost = orc.new_state()
    orc.run(ost, 320, threads=THREADS)
    assert np.all((st["N"] == 320) | (st["status"] != 0))
    cls = _classify(b, st, orc, ost, sc, counts, pairs)
    first = _check_switches(b, st, sc, cls, tp=tp)
    gpu_only, orc_flags = _flags(st, ost, range(8))
    print("320-link robots: %d match, %d switches (parting at steps %s), %d flagged (%d by the GPU alone)" % (
        cls.count("match"), cls.count("switch"), first, cls.count("flagged"), gpu_only))
    # along its own 320-step trajectory an FP32 robot can reach a state where
    # its step does not converge (Hessian condition numbers up to 2.5e7 on
    # these chains); from the oracle's states it does not (the long-chain
    # stepwise test: no GPU-only failure in 2179 robot-steps)
    assert gpu_only <= 2 and orc_flags == 0
    b.close()


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
    """4096 robots x 100 links in the launch the benchmark times (one-,
    two- and four-warp teams); 50 sampled robots recomputed by the oracle."""
    sc = scenes.design_batch()
    b = vine.Batch(sc, _prm(tp))
    b.simulate()
    torch.cuda.synchronize()
    st = b.state()
    counts, pairs = b.contacts(256)
    stats = b.stats()
    assert np.all((st["N"] == 100) | (st["status"] != 0))  # a failed step stops a robot
    nbad = int((st["status"] != 0).sum())
    # the FP64 oracle itself leaves about 0.5 % of these robots with a step
    # that does not converge in 100 iterations (deep-penetration coiling)
    assert nbad <= 40, "too many non-converged robots: %d" % nbad
    idx = np.sort(np.random.default_rng(7).choice(4096, 50, replace=False))
    sub = scenes.subset(sc, idx)
    orc = _oracle(sub)
    ost = orc.new_state()
    orc.run(ost, 100, threads=THREADS)
    cls = _classify(b, st, orc, ost, sub, counts, pairs, idx_gpu=idx)
    first = _check_switches(b, st, sub, cls, idx_gpu=idx, tp=tp)
    print("design batch sample: %d match, %d basin switches (parting at steps %s), %d flagged" % (
        cls.count("match"), cls.count("switch"), first, cls.count("flagged")))
    assert cls.count("flagged") <= 2
    assert stats["robot_link_steps"] >= 0.99 * scenes.robot_link_steps(sc["n_links"])
    b.close()


def test_uneven_batch_full_size_sampled():
    """The uneven batch at its full size (16 384 robots, links U{30..300},
    5-200 obstacles, 0-8 actuators) in one launch with the library's default
    launch configuration; 50 sampled robots recomputed by the oracle."""
    sc = scenes.uneven_batch()
    b = vine.Batch(sc)
    b.simulate()
    st = b.state()
    counts, pairs = b.contacts(1024)
    assert np.all((st["N"] == sc["n_links"]) | (st["status"] != 0))
    # some step of about 3.5 % of these robots runs out of iterations (the
    # oracle: 2 of the 50 sampled robots)
    assert int((st["status"] != 0).sum()) <= 0.05 * sc["n_links"].size
    idx = np.sort(np.random.default_rng(11).choice(sc["n_links"].size, 50, replace=False))
    sub = scenes.subset(sc, idx)
    orc = _oracle(sub)
    ost = orc.new_state()
    orc.run(ost, 300, threads=THREADS)
    cls = _classify(b, st, orc, ost, sub, counts, pairs, idx_gpu=idx)
    first = _check_switches(b, st, sub, cls, idx_gpu=idx)
    gpu_only, orc_flags = _flags(st, ost, idx)
    print("uneven sample: %d match, %d basin switches (parting at steps %s), %d flagged: %d by the GPU alone, "
          "%d by the oracle (links %d-%d)" % (cls.count("match"), cls.count("switch"), first, cls.count("flagged"),
                                             gpu_only, orc_flags, sub["n_links"].min(), sub["n_links"].max()))
    # some step of about 5 % of these robots runs out of iterations on either
    # side (FP64 oracle: 4 %); the FP32 kernel fails where the oracle does not
    # on at most 3 of the 50
    assert gpu_only <= 3
    b.close()


def test_robustness_batch_full_size_sampled():
    """The robustness batch at its full size (64 designs x 1024 perturbations,
    150 links, 60 obstacles) in one launch: forward poses and contact sets
    of 50 sampled robots against the oracle's growth."""
    sc, _goals = scenes.robustness_batch()
    b = vine.Batch(sc)
    b.simulate()
    st = b.state()
    counts, pairs = b.contacts(512)
    assert np.all((st["N"] == 150) | (st["status"] != 0))
    assert int((st["status"] != 0).sum()) <= 0.01 * sc["n_links"].size
    idx = np.sort(np.random.default_rng(13).choice(sc["n_links"].size, 50, replace=False))
    sub = scenes.subset(sc, idx)
    orc = _oracle(sub)
    ost = orc.new_state()
    orc.run(ost, 150, threads=THREADS)
    cls = _classify(b, st, orc, ost, sub, counts, pairs, idx_gpu=idx)
    first = _check_switches(b, st, sub, cls, idx_gpu=idx)
    print("robustness sample: %d match, %d basin switches (parting at steps %s), %d flagged" % (
        cls.count("match"), cls.count("switch"), first, cls.count("flagged")))
    assert cls.count("flagged") <= 2
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
    assert cls[0] == "match", cls
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
