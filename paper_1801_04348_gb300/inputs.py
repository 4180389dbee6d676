"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers (numpy's PCG64 `default_rng`); it holds
none of the GEMM's arithmetic.  Recipes:

* dense operands: A from `seed`, B from `seed + 1`; uniform[-1, 1] or normal(0, 1),
  float32, row-major;
* row scaling: every row multiplied by 10**u, u ~ uniform[-3, 3], drawn from its
  own seed (one factor per row of A and, separately, per row of B);
* integer-valued operands: integers drawn uniformly from [lo, hi], stored as float32;
* grouped shapes: M, N, K each log-uniform in [lo, hi], rounded to a multiple of 16
  and clamped to [lo, hi];
* cost-model weights: He-uniform U(-sqrt(6/fan_in), +sqrt(6/fan_in)), biases 0.
"""
from __future__ import annotations

import numpy as np


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape).astype(np.float32)


def normal(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=shape, dtype=np.float32)


def integers(shape, seed: int, lo: int = -4, hi: int = 4) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=shape).astype(np.float32)


def row_factors(rows: int, seed: int, decades: float = 3.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (10.0 ** rng.uniform(-decades, decades, size=rows)).astype(np.float32)


def gemm_operands(M: int, N: int, K: int, seed: int = 0, dist: str = "uniform"):
    """(A, B) with A: M x K from `seed`, B: K x N from `seed + 1`."""
    if dist == "uniform":
        return uniform((M, K), seed), uniform((K, N), seed + 1)
    if dist == "normal":
        return normal((M, K), seed), normal((K, N), seed + 1)
    if dist == "normal_rowscaled":
        A = normal((M, K), seed) * row_factors(M, seed + 100)[:, None]
        B = normal((K, N), seed + 1) * row_factors(K, seed + 101)[:, None]
        return A.astype(np.float32), B.astype(np.float32)
    if dist == "integers":
        return integers((M, K), seed), integers((K, N), seed + 1)
    raise ValueError(dist)


def log_uniform_dims(count: int, seed: int, lo: int, hi: int, multiple: int = 16) -> np.ndarray:
    """count x 3 int array of (M, N, K), each log-uniform in [lo, hi], rounded to
    `multiple` and clamped to [lo, hi]."""
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), size=(count, 3)))
    x = np.rint(x / multiple) * multiple
    return np.clip(x, lo, hi).astype(np.int64)


def he_uniform_mlp(seed: int = 0, d_in: int = 7, h: int = 64) -> np.ndarray:
    """Flat float32 parameter vector W1 (h x d_in), b1, W2 (h x h), b2, w3 (h), b3."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, size=(h, d_in)) * np.sqrt(6.0 / d_in)
    W2 = rng.uniform(-1, 1, size=(h, h)) * np.sqrt(6.0 / h)
    w3 = rng.uniform(-1, 1, size=(h,)) * np.sqrt(6.0 / h)
    return np.concatenate([W1.reshape(-1), np.zeros(h), W2.reshape(-1), np.zeros(h),
                           w3, np.zeros(1)]).astype(np.float32)
