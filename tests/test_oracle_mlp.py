"""Pins for the FP64 cost-model MLP oracle: central finite differences of the loss,
closed forms of degenerate networks, and Adam's first step."""
import numpy as np

from oracle import mlp
from paper_1801_04348_gb300 import inputs


def _data(B, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, 7)), rng.standard_normal(B)


def test_gradient_central_differences():
    theta = inputs.he_uniform_mlp(0).astype(np.float64)
    theta += np.random.default_rng(1).normal(0, 0.05, theta.size)   # non-zero biases
    X, t = _data(16, 2)
    _, g = mlp.loss_and_grad(theta, X, t)
    h = 1e-6
    rng = np.random.default_rng(3)
    idx = np.concatenate([np.arange(mlp.N_PARAMS - 200, mlp.N_PARAMS), rng.choice(mlp.N_PARAMS, 400, replace=False)])
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss(theta + e, X, t) - mlp.loss(theta - e, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_constant_network_closed_form():
    theta = np.zeros(mlp.N_PARAMS)
    theta[-1] = 0.75                              # b3
    X, t = _data(10, 4)
    y, _ = mlp.forward(theta, X)
    assert np.all(y == 0.75)
    L, g = mlp.loss_and_grad(theta, X, t)
    assert abs(L - np.mean((0.75 - t) ** 2)) < 1e-15
    assert abs(g[-1] - 2 * np.mean(0.75 - t)) < 1e-15
    assert np.all(g[:-1] == 0)


def test_linear_regime_closed_form():
    # all pre-activations positive -> the network is the affine map
    # y = w3 (W2 (W1 x + b1) + b2) + b3
    rng = np.random.default_rng(5)
    p = {"W1": rng.uniform(0, 1, (64, 7)), "b1": rng.uniform(0, 1, 64),
         "W2": rng.uniform(0, 1, (64, 64)), "b2": rng.uniform(0, 1, 64),
         "w3": rng.normal(0, 1, 64), "b3": np.array([0.3])}
    X = rng.uniform(0, 1, (9, 7))
    y, _ = mlp.forward(mlp.pack(p), X)
    want = (p["W2"] @ (p["W1"] @ X.T + p["b1"][:, None]) + p["b2"][:, None]).T @ p["w3"] + 0.3
    assert np.allclose(y, want, rtol=1e-13, atol=0)


def test_adam_first_step():
    rng = np.random.default_rng(6)
    theta = rng.normal(size=50)
    g = rng.normal(size=50)
    t1, m, v = mlp.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    # bias-corrected first step: mhat = g, vhat = g^2  ->  -lr g / (|g| + eps)
    assert np.allclose(t1 - theta, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
