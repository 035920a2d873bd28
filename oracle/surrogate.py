"""Oracle for the sPAM neural surrogate of Sec. 4.3: a 2-32-2 network with
ReLU hidden units (He initialisation) from the actuator strain and cell
length to the model parameters (m, phi_Rc), trained by mean squared error on
normalised outputs.

TEST INFRASTRUCTURE ONLY: the tests are the only users; the product package
never imports this module.  Plain float64 numpy, the formulas written out.

Layout shared with the library's surrogate (the order of the parameters in
one flat vector of 162):
  W1[32][2] (hidden j, input i), b1[32], W2[2][32] (output k, hidden j), b2[2].
Normalisation (constants chosen by the caller, part of the network):
  x_i = (input_i - in_lo_i) * in_scale_i;  output_k = y_k / out_scale_k.
Loss over n samples: L = (1 / (2 n)) sum_s sum_k (y_k - t_k)^2 with t the
normalised targets (t_k = target_k * out_scale_k).
Adam (Kingma and Ba 2015): beta1 0.9, beta2 0.999, eps 1e-8, step t counted
from 1, bias-corrected moments.
"""
from __future__ import annotations

import numpy as np

H = 32
N_PARAM = H * 2 + H + 2 * H + 2


def unpack(theta):
    th = np.asarray(theta, np.float64)
    W1 = th[0: 2 * H].reshape(H, 2)
    b1 = th[2 * H: 3 * H]
    W2 = th[3 * H: 5 * H].reshape(2, H)
    b2 = th[5 * H: 5 * H + 2]
    return W1, b1, W2, b2


def forward(theta, x):
    """Network outputs y[n, 2] for normalised inputs x[n, 2]."""
    W1, b1, W2, b2 = unpack(theta)
    a = np.asarray(x, np.float64) @ W1.T + b1
    h = np.maximum(a, 0.0)
    return h @ W2.T + b2


def loss_and_grad(theta, x, t):
    """(L, dL/dtheta) for normalised inputs x and targets t."""
    W1, b1, W2, b2 = unpack(theta)
    x = np.asarray(x, np.float64)
    n = x.shape[0]
    a = x @ W1.T + b1
    h = np.maximum(a, 0.0)
    y = h @ W2.T + b2
    r = y - np.asarray(t, np.float64)
    L = 0.5 * np.sum(r * r) / n
    dy = r / n                       # dL/dy
    gW2 = dy.T @ h
    gb2 = dy.sum(0)
    dh = dy @ W2
    da = dh * (a > 0.0)
    gW1 = da.T @ x
    gb1 = da.sum(0)
    return L, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2])


def adam(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def he_init(rng):
    """He initialisation: weights N(0, 2 / fan_in), biases zero."""
    W1 = rng.standard_normal((H, 2)) * np.sqrt(2.0 / 2)
    W2 = rng.standard_normal((2, H)) * np.sqrt(2.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(2)])
