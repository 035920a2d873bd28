"""The sPAM neural surrogate of Sec. 4.3, trained and evaluated in the
library's kernels.

The paper samples m in (0, 0.5] and l_0 in [0.02, 0.08] m, runs the exact
model for (strain, phi_Rc), and fits a 2-32-2 ReLU network (He
initialisation) from (strain, l_0) to (m, phi_Rc) on 40 000 samples split
80/10/10, reporting a mean squared error of 0.003 on normalised outputs.
``train`` does the same: seeded samples (m from the tabulated range
[m_lo, 0.5]), the exact model (``vine_spam_samples``), min-max input
normalisation and output scaling by the parameters' ranges (m / 0.5,
phi / (pi / 2)), full-batch Adam (``vine_surrogate_train``), and the
normalised mean squared error on the held-out parts (``vine_surrogate_eval``).
"""
from __future__ import annotations

import math

import numpy as np

from . import vine


def make_dataset(n: int = 40000, seed: int = 0, l0_range=(0.02, 0.08), params: vine.vine_params | None = None):
    """Samples of the exact model: inputs (strain, l0), targets (m, phi)."""
    p = params or vine.vine_params_default()
    rng = np.random.default_rng(seed)
    m = rng.uniform(p.m_lo, 0.5, n)
    l0 = rng.uniform(l0_range[0], l0_range[1], n)
    s = vine.spam_samples(m, l0, p)
    return np.stack([s["eps"], l0], 1), np.stack([m, s["phi"]], 1), s


def init_net(x_train: np.ndarray, seed: int = 0) -> dict:
    """He initialisation and the normalisation of the training inputs."""
    rng = np.random.default_rng(seed + 1)
    W1 = rng.standard_normal((32, 2)) * math.sqrt(2.0 / 2)
    W2 = rng.standard_normal((2, 32)) * math.sqrt(2.0 / 32)
    theta = np.concatenate([W1.ravel(), np.zeros(32), W2.ravel(), np.zeros(2)]).astype(np.float32)
    lo, hi = x_train.min(0), x_train.max(0)
    return dict(theta=theta, in_lo=lo.astype(np.float32), in_scale=(1.0 / (hi - lo)).astype(np.float32),
                out_scale=np.array([1.0 / 0.5, 1.0 / (0.5 * math.pi)], np.float32))


def normalised_mse(net: dict, x: np.ndarray, y: np.ndarray) -> float:
    """Mean squared error of the normalised outputs (the paper's measure)."""
    pred = vine.surrogate_eval(net, x)
    sc = np.asarray(net["out_scale"], np.float64)
    return float(np.mean(((pred - y) * sc) ** 2))


def train(n: int = 40000, steps: int = 3000, lr: float = 0.01, seed: int = 0, params=None) -> dict:
    """Data, split 80/10/10, training; returns the net, the loss history and
    the validation and test errors."""
    x, y, _ = make_dataset(n, seed, params=params)
    rng = np.random.default_rng(seed + 2)
    perm = rng.permutation(n)
    a, b = int(0.8 * n), int(0.9 * n)
    tr, va, te = perm[:a], perm[a:b], perm[b:]
    net = init_net(x[tr], seed)
    net, hist = vine.surrogate_train(net, x[tr], y[tr], steps, lr)
    return dict(net=net, history=hist, train_mse=normalised_mse(net, x[tr], y[tr]),
                val_mse=normalised_mse(net, x[va], y[va]), test_mse=normalised_mse(net, x[te], y[te]),
                x=x, y=y, split=(tr, va, te))
