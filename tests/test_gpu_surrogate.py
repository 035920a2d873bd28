"""sPAM surrogate (Sec. 4.3) on the GPU against the oracle
(oracle/surrogate.py and the FP64 sPAM model): training samples, the loss
and the first Adam steps from the same initial parameters, the network's
forward pass, and a full training run reaching the paper's accuracy."""
import numpy as np
import pytest

import oracle
from oracle import surrogate as osg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import surrogate, vine  # noqa: E402


def test_samples_match_the_oracle_model():
    rng = np.random.default_rng(4)
    m = np.concatenate([rng.uniform(0.002, 0.5, 300), [0.5, 0.002]])
    l0 = rng.uniform(0.02, 0.08, m.size)
    g = vine.spam_samples(m, l0)
    p = oracle.default_params()
    for i in range(m.size):
        e, f, ph, sat = oracle.spam_eval(m[i], l0[i], p)
        assert g["eps"][i] == pytest.approx(e, rel=1e-9, abs=1e-12), i
        assert g["phi"][i] == pytest.approx(ph, rel=1e-9), i
        assert g["f"][i] == pytest.approx(f, rel=1e-9, abs=1e-15), i
        assert bool(g["saturated"][i]) == sat, i


def _small(seed=0, n=2000):
    x, y, _ = surrogate.make_dataset(n, seed)
    net = surrogate.init_net(x, seed)
    return x, y, net


def _normed(net, x, y):
    xn = (x.astype(np.float32) - net["in_lo"]) * net["in_scale"]
    tn = y.astype(np.float32) * net["out_scale"]
    return xn.astype(np.float64), tn.astype(np.float64)


def test_loss_and_adam_steps_match_the_oracle():
    x, y, net = _small()
    xn, tn = _normed(net, x, y)
    th = net["theta"].astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    losses = []
    for s in range(1, 4):
        L, g = osg.loss_and_grad(th, xn, tn)
        losses.append(L)
        th, m, v = osg.adam(th, g, m, v, s, 0.01)
    got, hist = vine.surrogate_train(net, x, y, 3, 0.01)
    assert np.allclose(hist, losses, rtol=1e-5, atol=0)
    assert np.allclose(got["theta"], th, rtol=1e-4, atol=2e-6), np.max(np.abs(got["theta"] - th))


def test_forward_matches_the_oracle_and_training_is_deterministic():
    x, y, net = _small(1)
    a, _ = vine.surrogate_train(net, x, y, 50, 0.01, history=False)
    b, _ = vine.surrogate_train(net, x, y, 50, 0.01, history=False)
    assert np.array_equal(a["theta"], b["theta"])
    xn, _ = _normed(a, x, y)
    ref = osg.forward(a["theta"].astype(np.float64), xn) / a["out_scale"].astype(np.float64)
    got = vine.surrogate_eval(a, x)
    assert np.allclose(got, ref, rtol=1e-5, atol=1e-6)
    dev = vine.surrogate_eval(a, torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), got)


def test_full_training_reaches_the_papers_accuracy():
    r = surrogate.train(40000, steps=3000, lr=0.01)
    h = r["history"]
    print("surrogate: loss %.4g -> %.4g; normalised MSE train %.4g val %.4g test %.4g (paper: 0.003)"
          % (h[0], h[-1], r["train_mse"], r["val_mse"], r["test_mse"]))
    assert h[-1] < 0.2 * h[0]
    assert r["test_mse"] <= 0.01
    assert abs(r["val_mse"] - r["test_mse"]) <= 0.5 * max(r["val_mse"], r["test_mse"])
