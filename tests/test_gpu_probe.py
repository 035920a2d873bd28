"""GPU parity of one evaluation: at fixed states taken from the oracle's own
trajectories (rounded to float32), the CUDA cost, gradient, Gauss-Newton step
and its residual against the FP64 oracle's."""
import numpy as np
import pytest

import oracle
from paper_2509_15180_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402


def _displacements(orc, i, th, l, dx):
    """Displacement of every link end predicted by the step dx (joint angles, then l)."""
    px, py, psi = orc.poses(i, th, l)
    N = th.size
    out = np.zeros((N, 2))
    for k in range(N):
        rx, ry = px[k + 1] - px[: k + 1], py[k + 1] - py[: k + 1]
        out[k, 0] = np.sum(-dx[: k + 1] * ry)
        out[k, 1] = np.sum(dx[: k + 1] * rx)
    out[N - 1] += dx[N] * np.array([np.cos(psi[N - 1]), np.sin(psi[N - 1])])
    return out


def _states(sc, steps, every):
    orc = oracle.Oracle(sc, oracle.default_params(tol=1e-10))
    st = orc.new_state()
    out = []
    for s in range(steps):
        orc.run(st, 1, threads=8)
        if (s + 1) % every == 0:
            for i in range(sc["n_links"].size):
                out.append((i, orc.theta_of(st, i).astype(np.float32), np.float32(st["l"][i])))
    return orc, out


@pytest.mark.parametrize("batch", ["parity", "design"])
@pytest.mark.parametrize("exact", [0, 1])
def test_probe_matches_oracle(batch, exact):
    """Gauss-Newton mode checks the O(N) sweep at every state, including
    states pushed off equilibrium; exact-Hessian mode at the equilibrium
    states only (off equilibrium the exact Hessian can be near singular,
    where FP32 and FP64 steps legitimately part)."""
    sc = scenes.parity_batch(16) if batch == "parity" else scenes.design_batch(8)
    steps, every = (20, 5) if batch == "parity" else (60, 15)
    orc, states = _states(sc, steps, every)
    orc = oracle.Oracle(sc, oracle.default_params(exact_hessian=exact))
    prm = vine.vine_params_default()
    prm.exact_hessian = exact
    b = vine.Batch(sc, prm)
    worst = dict(J=0.0, g=0.0, dx=0.0, r=0.0)
    for (i, th, l) in states:
        th64 = th.astype(np.float64)
        # perturb off the equilibrium so the gradient and step are not ~0
        pert = th64 + 1e-3 * np.sin(np.arange(th.size) * 1.7 + i)
        cases = ((th64, float(l)), (pert, float(l) * 0.7)) if not exact else ((th64, float(l)),)
        for thv, lv in cases:
            th32 = thv.astype(np.float32)
            Jg, gg, dg, rg, lfg = b.probe(i, th32, lv)
            dxo, ro, Jo, lfo = orc.gn_step(i, th32.astype(np.float64), float(np.float32(lv)))
            _, go, _ = orc.energy(i, th32.astype(np.float64), float(np.float32(lv)), hessian=False)
            assert lfg == lfo
            # J can nearly cancel (bending vs actuator energy); scale by one
            # joint's onset energy w_a pi P R^3 as well
            scale = abs(Jo) + 160.0 * np.pi * float(sc["pressure"][i]) * float(sc["radius"][i]) ** 3
            worst["J"] = max(worst["J"], abs(Jg - Jo) / scale)
            # at equilibrium states the gradient and step are ~0: compare
            # against the joint moment scale and a 1e-4 rad step scale too
            worst["g"] = max(worst["g"], np.max(np.abs(gg - go)) / (np.max(np.abs(go)) + scale))
            # compare the steps as the link-end displacements they predict (the
            # soft directions of an ill-conditioned matrix are resolved only
            # to FP32 accuracy in joint-angle terms)
            th_o = th32.astype(np.float64)
            dg_p = _displacements(orc, i, th_o, float(np.float32(lv)), dg.astype(np.float64))
            do_p = _displacements(orc, i, th_o, float(np.float32(lv)), dxo)
            # in link lengths: at an equilibrium state both steps are FP32/FP64
            # noise, so the bar is the pose tolerance (1e-4 link lengths) plus
            # 1% of the step
            ls = float(sc["l_seg"][i])
            e = np.max(np.abs(dg_p - do_p)) / (1e-4 * ls + 1e-2 * np.max(np.abs(do_p)))
            key = "dx" if thv is th64 else "dx_off"
            worst[key] = max(worst.get(key, 0.0), e)
            # the residual is relative to the robot length and tested against
            # tol = 1e-6: at equilibrium both sides read FP32/FP64 noise of
            # about that size, so the bar is tol plus 2% of the residual
            worst["r"] = max(worst["r"], abs(rg - ro) / (1e-6 + 2e-2 * ro))
    print("probe %s batch, exact %d, worst relative errors: %s" % (batch, exact, worst))
    # FP32 terms and the Hermite-tabulated wrinkling energy near onset
    assert worst["J"] < 1e-4
    assert worst["g"] < 5e-3  # FP32 contact forces: ~1e-8 m penetration error x stiffness x lever
    assert worst["dx"] < 1.0
    assert worst.get("dx_off", 0.0) < 1.0
    assert worst["r"] < 1.0
    b.close()
