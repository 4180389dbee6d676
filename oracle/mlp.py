"""Cost-model MLP in binary64 -- TEST INFRASTRUCTURE ONLY.

The learned cost model ranks feasible program parameters (the paper leaves the
choice of program parameters to auto-tuning, Section 1).  Its network is
7 -> 64 -> 64 -> 1 with ReLU after each hidden layer:

    z1 = W1 x + b1,  h1 = relu(z1)
    z2 = W2 h1 + b2, h2 = relu(z2)
    y  = w3 . h2 + b3

trained with the mean squared error L = (1/B) sum_b (y_b - t_b)^2 and Adam
(Kingma & Ba 2015: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
theta <- theta - lr * mhat / (sqrt(vhat) + eps), mhat = m/(1-b1^t),
vhat = v/(1-b2^t)).  relu'(z) is taken as 1 for z > 0 and 0 otherwise.

Parameters travel as one flat vector in the order W1 (64x7 row-major), b1 (64),
W2 (64x64 row-major), b2 (64), w3 (64), b3 (1): 4737 values.
"""
from __future__ import annotations

import numpy as np

D_IN, H = 7, 64
SHAPES = [("W1", (H, D_IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
          ("w3", (H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    out, off = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[off:off + n].reshape(shape)
        off += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1)
                           for name, _ in SHAPES])


def forward(theta: np.ndarray, X: np.ndarray):
    """Return y (B,) and the intermediates (z1, h1, z2, h2)."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.where(z1 > 0, z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.where(z2 > 0, z2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (z1, h1, z2, h2)


def loss(theta: np.ndarray, X: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(theta, X)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def loss_and_grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray):
    """Mean squared error and its gradient by the chain rule (backpropagation)."""
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    p = unpack(theta)
    y, (z1, h1, z2, h2) = forward(theta, X)
    B = X.shape[0]
    r = y - t
    L = float(np.mean(r ** 2))
    dy = 2.0 * r / B                        # dL/dy_b
    g = {}
    g["w3"] = h2.T @ dy
    g["b3"] = np.array([np.sum(dy)])
    dz2 = np.outer(dy, p["w3"]) * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return L, pack(g)


def adam_step(theta, grad, m, v, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1).  Returns new (theta, m, v)."""
    theta = np.asarray(theta, dtype=np.float64)
    grad = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v
