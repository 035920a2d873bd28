"""GPU adjoint (vine_grad) against the FP64 oracle's adjoint at the same
state (the oracle's equilibria, loaded into the GPU batch), the actuator
update path, and the torch.autograd.Function."""
import numpy as np
import pytest

import oracle
from paper_2509_15180_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402
from paper_2509_15180_gb300.autograd import VineSim  # noqa: E402


def _scene(n_designs=6, n_perturb=2, n_links=30):
    return scenes.robustness_batch(n_designs=n_designs, n_perturb=n_perturb, n_links=n_links, box=0.015 * n_links,
                          n_circ=8, n_box=8)


def _cond(orc, i, th, l):
    """2-norm condition number of the exact Hessian on the free unknowns (the
    distal length dropped when its bound is active, as in the solver)."""
    H = orc.hessian_exact(i, th, l)
    _, g, _ = orc.energy(i, th, l, hessian=False)
    ls = float(orc._keep["l_seg"][i])
    lfix = (l <= 0.0 and g[-1] > 0.0) or (l >= ls and g[-1] < 0.0)
    if lfix:
        H = H[:-1, :-1]
    w = np.abs(np.linalg.eigvalsh(0.5 * (H + H.T)))
    return float(w.max() / max(w.min(), 1e-300))


def _oracle_equilibria(sc):
    """The oracle's growth of every robot to full length, rounded to FP32 (the
    GPU's storage precision): the states at which both adjoints are taken."""
    orc = oracle.Oracle(sc)
    ost = orc.new_state()
    orc.run(ost, int(sc["n_links"].max()), threads=16)
    ost["theta"][:] = ost["theta"].astype(np.float32)
    ost["l"][:] = ost["l"].astype(np.float32)
    return orc, ost


def _load(b, sc, orc, ost, idx=None, base=None):
    """vine_set_state with the oracle's states: robot idx[j] of the GPU batch
    gets the oracle's robot j; the others keep the state `base` (a state()
    of the batch itself)."""
    n = sc["n_links"].size
    idx = np.arange(n) if idx is None else np.asarray(idx)
    if base is None:
        N = np.zeros(n, np.int32)
        th = np.zeros(max(b.total_links, 1), np.float32)
        l = np.zeros(n, np.float32)
    else:
        N, th, l = base["N"].copy(), base["theta"].copy(), base["l"].copy()
    for j, i in enumerate(idx):
        N[i] = ost["N"][j]
        th[b.offsets[i]: b.offsets[i] + N[i]] = orc.theta_of(ost, j)
        l[i] = ost["l"][j]
    b.set_state(N, th, l)


REL = 1e-2        # per-derivative relative bar
FLOOR = 1e-3      # absolute floor: this fraction of the largest derivative of its kind in the sample
COND_MAX = 1e7    # robots whose exact Hessian is worse conditioned are counted, not compared


def _compare(sc, orc, ost, goals, g, min_checked, idx=None, kind="tip", paths=None):
    """GPU adjoint against the FP64 oracle's at the same state (the oracle's
    own equilibrium rounded to FP32, loaded with vine_set_state).  Oracle
    robot j is GPU robot idx[j].  Bar per derivative: REL of itself plus
    FLOOR of the largest derivative of its kind (some are ~0: an actuator
    whose moment barely reaches the cost).  The FP32 Hessian carries
    relative errors of ~6e-8 per entry, which move lambda = H^-1 c by up to
    cond x 6e-8: robots whose condition number exceeds COND_MAX are counted
    and bounded, not compared."""
    idx = np.arange(orc.n) if idx is None else np.asarray(idx)
    off = np.concatenate([[0], np.cumsum(sc["n_links"])])
    rows = []
    skipped = ill = 0
    conds = {}
    for j, i in enumerate(idx):
        a0, a1 = int(sc["act_ptr"][i]), int(sc["act_ptr"][i + 1])
        if ost["status"][j] != 0 or g["status"][i] != 0:
            skipped += 1
            continue
        th, l = orc.theta_of(ost, j), float(ost["l"][j])
        if kind == "tip":
            c, dP, dB, dE, rc = orc.grad(j, th, l, goals[i].astype(np.float64))
        else:
            c, dP, dB, dE, rc = orc.grad_path(j, th, l, paths[off[i]: off[i + 1]].astype(np.float64))
        if rc != 0:
            skipped += 1
            continue
        assert abs(g["cost"][i] - c) <= 1e-5 * max(c, 1e-6), (i, g["cost"][i], c)
        conds[i] = _cond(orc, j, th, l)
        if conds[i] > COND_MAX:
            ill += 1
            continue
        for k, v in (("dP", dP), ("dB", dB), ("dE", dE)):
            for a in range(a1 - a0):
                rows.append((k, i, a, g[k][a0 + a], v[a]))
    worst = {}
    for k in ("dP", "dB", "dE"):
        sel = [r for r in rows if r[0] == k]
        if not sel:
            continue
        scale = max(abs(r[4]) for r in sel)
        errs = [abs(r[3] - r[4]) / (REL * abs(r[4]) + FLOOR * scale) for r in sel]
        worst[k] = max(errs)
        q = int(np.argmax(errs))
        assert worst[k] < 1.0, (k, worst[k], sel[q], "cond %.3g" % conds[sel[q][1]])
    cv = np.array(list(conds.values())) if conds else np.zeros(1)
    print("%s-cost adjoint parity: %d derivatives, %d robots skipped, %d of %d beyond cond %.0e; worst (fraction "
          "of the bar) %s; condition numbers median %.3g, max compared %.3g" % (
              kind, len(rows), skipped, ill, len(conds), COND_MAX, worst, float(np.median(cv)),
              float(cv[cv <= COND_MAX].max()) if np.any(cv <= COND_MAX) else 0.0))
    assert ill <= 0.25 * max(len(conds), 1)
    assert len(rows) >= min_checked
    return worst


def test_grad_matches_oracle_adjoint_small():
    sc, goals = _scene()
    orc, ost = _oracle_equilibria(sc)
    b = vine.Batch(sc)
    _load(b, sc, orc, ost)
    g = b.grad(goals)
    _compare(sc, orc, ost, goals, g, 40)
    b.close()


def test_path_grad_matches_oracle_adjoint():
    """The path cost (1/N) sum_k |p_k - q_k|^2 against the oracle's adjoint,
    on the small robots and on 150-link robots of the robustness designs."""
    sc, goals = _scene()
    paths = scenes.goal_paths(sc, goals)
    orc, ost = _oracle_equilibria(sc)
    b = vine.Batch(sc)
    _load(b, sc, orc, ost)
    g = b.grad_path(paths)
    _compare(sc, orc, ost, goals, g, 40, kind="path", paths=paths)
    b.close()
    sc, goals = scenes.robustness_batch(n_designs=8, n_perturb=3)
    paths = scenes.goal_paths(sc, goals)
    orc, ost = _oracle_equilibria(sc)
    b = vine.Batch(sc)
    _load(b, sc, orc, ost)
    g = b.grad_path(paths)
    _compare(sc, orc, ost, goals, g, 20, kind="path", paths=paths)
    b.close()


def test_grad_device_path_equals_host_path():
    sc, goals = _scene(4, 2)
    b = vine.Batch(sc)
    b.simulate()
    gh = b.grad(goals)
    gd = b.grad(torch.from_numpy(goals).cuda())
    torch.cuda.synchronize()
    for k in ("cost", "dP", "dB", "dE", "status"):
        assert np.array_equal(gd[k].cpu().numpy(), gh[k], equal_nan=True), k
    b.close()


def test_grad_full_length_robustness_designs_sampled():
    """Robustness-batch designs at full size (150 links, 60 obstacles, 2.25 m
    box), 8 designs x 16 perturbations grown in one launch; then 24 sampled
    robots are set to the oracle's equilibria and the adjoint of the whole
    batch is taken in one launch, the sampled robots checked against the
    oracle's adjoint."""
    sc, goals = scenes.robustness_batch(n_designs=8, n_perturb=16)
    b = vine.Batch(sc)
    b.simulate()
    st = b.state()
    g = b.grad(goals)
    ok = (g["status"] == 0) & (st["status"] == 0)
    print("robots with a gradient: %d of %d (status %s)" % (ok.sum(), ok.size, np.bincount(g["status"])))
    assert ok.mean() >= 0.8
    idx = np.sort(np.random.default_rng(3).choice(len(goals), 24, replace=False))
    orc, ost = _oracle_equilibria(scenes.subset(sc, idx))
    _load(b, sc, orc, ost, idx=idx, base=st)
    g = b.grad(goals)
    _compare(sc, orc, ost, goals, g, 30, idx=idx)
    b.close()


def test_set_actuators_equals_fresh_batch():
    sc, goals = _scene(4, 2)
    rng = np.random.default_rng(11)
    p2 = (sc["act_pressure"] * rng.uniform(0.8, 1.2, sc["act_pressure"].size)).astype(np.float32)
    b2 = (sc["act_begin"] + rng.uniform(-0.3, 0.3, sc["act_begin"].size)).clip(0.0).astype(np.float32)
    e2 = np.maximum(sc["act_end"] + rng.uniform(-0.3, 0.3, sc["act_end"].size), b2 + 0.5).astype(np.float32)
    ref = dict(sc, act_pressure=p2, act_begin=b2, act_end=e2)
    b = vine.Batch(sc)
    b.set_actuators(p2, b2, e2)
    b.reset()
    b.simulate()
    fresh = vine.Batch(ref)
    fresh.simulate()
    s1, s2 = b.state(), fresh.state()
    for k in ("theta", "l", "N", "status", "iters"):
        assert np.array_equal(s1[k], s2[k]), k
    # an invalid span marks only its robot
    bad_e = e2.copy()
    bad_e[0] = b2[0] - 1.0
    b.set_actuators(p2, b2, bad_e)
    b.reset()
    st = b.state()
    owner = int(np.searchsorted(sc["act_ptr"], 0, side="right") - 1)
    assert st["status"][owner] == vine.INST_BADINPUT
    assert np.all(np.delete(st["status"], owner) == 0)
    b.close(); fresh.close()


def test_autograd_function_chain_rule():
    sc, goals = _scene(4, 2)
    b = vine.Batch(sc)
    dev = torch.device("cuda")
    P = torch.tensor(sc["act_pressure"], device=dev, requires_grad=True)
    B = torch.tensor(sc["act_begin"], device=dev, requires_grad=True)
    E = torch.tensor(sc["act_end"], device=dev, requires_grad=True)
    goal = torch.tensor(goals, device=dev)
    cost = VineSim.apply(P, B, E, b, goal)
    w = torch.linspace(0.5, 2.0, cost.numel(), device=dev, dtype=torch.float64)
    (cost * w).sum().backward()
    g = b.grad(goals)
    owner = np.repeat(np.arange(len(goals)), np.diff(sc["act_ptr"]))
    wn = w.cpu().numpy()[owner]
    ok = ~np.isnan(g["dP"])
    assert np.allclose(P.grad.cpu().numpy()[ok], (wn * g["dP"])[ok].astype(np.float32), rtol=1e-6, atol=0)
    assert np.allclose(B.grad.cpu().numpy()[ok], (wn * g["dB"])[ok].astype(np.float32), rtol=1e-6, atol=0)
    assert np.allclose(E.grad.cpu().numpy()[ok], (wn * g["dE"])[ok].astype(np.float32), rtol=1e-6, atol=0)
    assert np.allclose(cost.detach().cpu().numpy(), g["cost"], rtol=0, atol=0)
    # the path cost through the same Function
    paths = scenes.goal_paths(sc, goals)
    for t in (P, B, E):
        t.grad = None
    cost = VineSim.apply(P, B, E, b, torch.tensor(paths, device=dev), "path")
    cost.sum().backward()
    gp = b.grad_path(paths)
    ok = ~np.isnan(gp["dP"])
    assert np.allclose(P.grad.cpu().numpy()[ok], gp["dP"][ok].astype(np.float32), rtol=1e-6, atol=0)
    assert np.allclose(cost.detach().cpu().numpy(), gp["cost"], rtol=0, atol=0)
    b.close()
