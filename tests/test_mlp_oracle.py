"""Pins of the FP64 cost-model oracle: gradients against central finite
differences, a case with a closed form, and Adam's first step."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    d, h = 7, 9
    rng = np.random.default_rng(0)
    theta = mlp.init(d, h, seed=1) + 0.01 * rng.standard_normal(mlp.n_params(d, h))
    X = rng.standard_normal((33, d))
    T = rng.standard_normal(33)
    L, g = mlp.loss_and_grad(theta, X, T, d, h)
    idx = rng.choice(len(theta), 60, replace=False)
    eps = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        fd = (mlp.loss_and_grad(tp, X, T, d, h)[0] - mlp.loss_and_grad(tm, X, T, d, h)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_linear_regime_closed_form():
    # all pre-activations positive: the network is affine, y = x A + c with
    # A = W1 W2 W3 and c = (b1 W2 + b2) W3 + b3
    d, h = 3, 4
    rng = np.random.default_rng(2)
    W1 = np.abs(rng.standard_normal((d, h))); b1 = np.abs(rng.standard_normal(h))
    W2 = np.abs(rng.standard_normal((h, h))); b2 = np.abs(rng.standard_normal(h))
    W3 = rng.standard_normal((h, 1)); b3 = rng.standard_normal(1)
    theta = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    X = np.abs(rng.standard_normal((10, d)))
    y, _ = mlp.forward(theta, X, d, h)
    A = W1 @ W2 @ W3
    c = (b1 @ W2 + b2) @ W3 + b3
    np.testing.assert_allclose(y, (X @ A + c)[:, 0], rtol=1e-13)


def test_adam_first_step_is_signed_lr():
    # t = 1: mhat = g, vhat = g^2, so the step is lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.1)
    np.testing.assert_allclose(th, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_training_reduces_loss():
    d, h = 5, 16
    rng = np.random.default_rng(4)
    X = rng.standard_normal((256, d))
    T = np.sin(X[:, 0]) + 0.5 * X[:, 1] ** 2
    theta = mlp.init(d, h, seed=3)
    m = np.zeros_like(theta); v = np.zeros_like(theta)
    L0 = mlp.loss_and_grad(theta, X, T, d, h)[0]
    for t in range(1, 301):
        L, g = mlp.loss_and_grad(theta, X, T, d, h)
        theta, m, v = mlp.adam_step(theta, g, m, v, t, lr=1e-2)
    assert L < 0.2 * L0
