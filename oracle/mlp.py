"""FP64 oracle of the plan cost model: a small multilayer perceptron
x -> ReLU(x W1 + b1) -> ReLU(. W2 + b2) -> . W3 + b3 (one output, the log of
a predicted time), mean-squared-error loss, and Adam (Kingma & Ba 2015:
beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected moments).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy, FP64, the
definitions written out layer by layer.

Parameters travel as one flat vector in the order
W1 (d_in x h, row-major), b1 (h), W2 (h x h), b2 (h), W3 (h x 1), b3 (1).
"""
from __future__ import annotations

import numpy as np


def sizes(d_in: int, h: int):
    return [(d_in, h), (h,), (h, h), (h,), (h, 1), (1,)]


def n_params(d_in: int, h: int) -> int:
    return sum(int(np.prod(s)) for s in sizes(d_in, h))


def unpack(theta: np.ndarray, d_in: int, h: int):
    out, o = [], 0
    for s in sizes(d_in, h):
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    return out


def forward(theta, X, d_in, h):
    """Returns y (rows,) and the cache of pre-activations."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, dtype=np.float64), d_in, h)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1 + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2 + b2
    a2 = np.maximum(z2, 0.0)
    y = (a2 @ W3 + b3)[:, 0]
    return y, (X, z1, a1, z2, a2)


def loss_and_grad(theta, X, T, d_in, h):
    """L = mean((y - t)^2) and dL/dtheta (flat), by the chain rule."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, dtype=np.float64), d_in, h)
    y, (X, z1, a1, z2, a2) = forward(theta, X, d_in, h)
    R = len(y)
    r = y - np.asarray(T, dtype=np.float64)
    L = float(np.mean(r * r))
    dy = (2.0 / R) * r[:, None]                 # dL/dy
    gW3 = a2.T @ dy
    gb3 = dy.sum(axis=0)
    da2 = dy @ W3.T
    dz2 = da2 * (z2 > 0)
    gW2 = a1.T @ dz2
    gb2 = dz2.sum(axis=0)
    da1 = dz2 @ W2.T
    dz1 = da1 * (z1 > 0)
    gW1 = X.T @ dz1
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def init(d_in, h, seed):
    """He-style normal initialisation (std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in sizes(d_in, h):
        if len(s) == 2:
            parts.append(rng.standard_normal(s).ravel() * np.sqrt(2.0 / s[0]))
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)
