"""The cost model's GPU kernels against the FP64 oracle (oracle/mlp.py):
forward values, loss gradients (relative error <= 1e-4 in FP32), the Adam
trajectory, and the host feature rows the planner feeds it."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1805_00988_gb300 import circuits as C


def test_feature_rows_cpu():
    from paper_1805_00988_gb300 import sim
    g = sim.to_sim_gates(C.haar_cz(20, 3, seed=1))
    rows = [sim.sim_plan_features(20, 0, g, v) for v in range(sim.N_VARIANTS)]
    for v, r in enumerate(rows):
        assert r is not None and r.shape == (sim.N_FEATURES,)
        assert r[6 + v] == 1.0 and np.sum(r[6:13]) == 1.0
    # fused needs complex64 and n >= k + 7; 12-qubit tiles need n >= 12
    assert sim.sim_plan_features(20, 1, g, 5) is None
    small = sim.to_sim_gates(C.qft(9))
    assert sim.sim_plan_features(9, 0, small, 1) is None
    assert sim.sim_plan_features(9, 0, small, 0) is not None


@pytest.fixture(scope="module")
def gsim():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1805_00988_gb300 import sim as S
    return S


def data(seed, rows=300, d=16):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, d)).astype(np.float32)
    T = (np.sin(X[:, 0]) + 0.3 * X[:, 1] * X[:, 2]).astype(np.float32)
    return X, T


@pytest.mark.gpu
def test_forward_and_gradient_vs_oracle(gsim):
    d, h = 16, 64
    X, T = data(1)
    theta = omlp.init(d, h, seed=2)
    m = gsim.MLP(d, h)
    m.set_params(theta.astype(np.float32))
    th32 = theta.astype(np.float32).astype(np.float64)
    y_ref, _ = omlp.forward(th32, X.astype(np.float64), d, h)
    np.testing.assert_allclose(m.forward(X), y_ref, rtol=1e-4, atol=1e-5)
    L, g = m.loss_grad(X, T)
    L_ref, g_ref = omlp.loss_and_grad(th32, X.astype(np.float64), T.astype(np.float64), d, h)
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert rel <= 1e-4, rel
    m.close()


@pytest.mark.gpu
def test_adam_trajectory_vs_oracle(gsim):
    d, h = 16, 32
    X, T = data(3, rows=200)
    theta = omlp.init(d, h, seed=4)
    m = gsim.MLP(d, h)
    m.set_params(theta.astype(np.float32))
    lr = 3e-3
    m.train(X, T, steps=20, lr=lr)
    th = theta.astype(np.float32).astype(np.float64)
    mm = np.zeros_like(th)
    vv = np.zeros_like(th)
    for t in range(1, 21):
        _, g = omlp.loss_and_grad(th, X.astype(np.float64), T.astype(np.float64), d, h)
        th, mm, vv = omlp.adam_step(th, g, mm, vv, t, lr)
    got = m.get_params().astype(np.float64)
    assert np.max(np.abs(got - th)) <= 2e-4, np.max(np.abs(got - th))
    m.close()


@pytest.mark.gpu
def test_training_fits(gsim):
    d, h = 16, 64
    X, T = data(5, rows=1000)
    m = gsim.MLP(d, h)
    m.set_params(omlp.init(d, h, seed=6).astype(np.float32))
    L0, _ = m.loss_grad(X, T)
    L = m.train(X, T, steps=400, lr=3e-3)
    assert L < 0.1 * L0
    m.close()
