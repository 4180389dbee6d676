"""Pins for the FP64 GEMM oracle (definition of Fig. "metamul"/"cudamul", Section 2).

Each test fixes the oracle against something other than itself: exact integer
arithmetic, closed forms, a long-double textbook loop, or numpy's BLAS product.
"""
import numpy as np
import pytest

from paper_1801_04348_gb300 import inputs


def test_integer_exact_bruteforce(oracle_mod):
    # Python integers are exact: C[i][j] = sum_k A[i][k] B[k][j], non-square so a
    # transposed operand or swapped index cannot pass.
    A = inputs.integers((7, 5), 3)
    B = inputs.integers((5, 9), 4)
    C = oracle_mod.gemm(A, B)
    for i in range(7):
        for j in range(9):
            want = sum(int(A[i, k]) * int(B[k, j]) for k in range(5))
            assert C[i, j] == want


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (3, 2, 7), (9, 9, 9), (4, 8, 1), (1, 9, 5)])
def test_against_longdouble(oracle_mod, M, N, K):
    A, B = inputs.gemm_operands(M, N, K, seed=M * 100 + N * 10 + K)
    C = oracle_mod.gemm(A, B)
    Cl = oracle_mod.gemm_longdouble(A, B)
    # forward error bound of a length-K binary64 dot product: K u |A||B|
    bound = K * 2.0 ** -53 * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64))
    assert np.all(np.abs(C - Cl) <= bound * 1.01 + 1e-300)


def test_identity_and_ones(oracle_mod):
    B = inputs.uniform((6, 11), 5)
    assert np.array_equal(oracle_mod.gemm(np.eye(6, dtype=np.float32), B), B.astype(np.float64))
    K = 37
    C = oracle_mod.gemm(np.ones((4, K), np.float32), np.ones((K, 5), np.float32))
    assert np.all(C == K)


def test_rank1_closed_form(oracle_mod):
    # A = x y^T, B = y' z^T  ->  C = (y . y') x z^T
    x = np.array([1.0, -2.0, 0.5], np.float32)
    y = np.array([2.0, 1.0, -1.0, 4.0], np.float32)
    yp = np.array([0.5, -3.0, 2.0, 1.0], np.float32)
    z = np.array([1.0, 2.0, -4.0, 0.25, 8.0], np.float32)
    A = np.outer(x, y).astype(np.float32)
    B = np.outer(yp, z).astype(np.float32)
    C = oracle_mod.gemm(A, B)
    want = float(np.dot(y.astype(np.float64), yp.astype(np.float64))) * np.outer(x, z)
    assert np.array_equal(C, want)


def test_beta_accumulate_and_rows(oracle_mod):
    A, B = inputs.gemm_operands(13, 17, 19, seed=2)
    AB = oracle_mod.gemm(A, B)
    C0 = inputs.uniform((13, 17), 9).astype(np.float64)
    C1 = oracle_mod.gemm(A, B, C0=C0, beta=1.0)
    assert np.allclose(C1, C0 + AB, rtol=0, atol=1e-13)
    # beta = 1 with C0 = -A B cancels (paper's accumulate form c += a b)
    Z = oracle_mod.gemm(A, B, C0=-AB, beta=1.0)
    assert np.max(np.abs(Z)) < 1e-13
    rows = np.array([12, 0, 5, 5])
    assert np.array_equal(oracle_mod.gemm(A, B, rows=rows), AB[rows])


def test_against_numpy_blas(oracle_mod):
    A, B = inputs.gemm_operands(64, 80, 96, seed=7)
    C = oracle_mod.gemm(A, B)
    ref = A.astype(np.float64) @ B.astype(np.float64)
    assert oracle_mod.rel_frobenius(C, ref) < 1e-14


def test_rel_frobenius_closed_forms(oracle_mod):
    X = inputs.uniform((5, 6), 1).astype(np.float64)
    assert oracle_mod.rel_frobenius(X, X) == 0.0
    assert abs(oracle_mod.rel_frobenius(2 * X, X) - 1.0) < 1e-15
    assert abs(oracle_mod.rel_frobenius(np.zeros_like(X), X) - 1.0) < 1e-15


def _wrap32(x):
    x %= 2 ** 32
    return x - 2 ** 32 if x >= 2 ** 31 else x


def test_int32_oracle_against_python_integers(oracle_mod):
    # full-range int32 values: products and sums overflow, exact Python integers
    # reduced modulo 2^32 give the two's-complement result
    rng = np.random.default_rng(11)
    A = rng.integers(-2 ** 31, 2 ** 31, size=(5, 9), dtype=np.int64).astype(np.int32)
    B = rng.integers(-2 ** 31, 2 ** 31, size=(9, 4), dtype=np.int64).astype(np.int32)
    C0 = rng.integers(-2 ** 31, 2 ** 31, size=(5, 4), dtype=np.int64).astype(np.int32)
    C = oracle_mod.gemm_i32(A, B)
    C1 = oracle_mod.gemm_i32(A, B, C0=C0, beta=1)
    for i in range(5):
        for j in range(4):
            exact = sum(int(A[i, k]) * int(B[k, j]) for k in range(9))
            assert C[i, j] == _wrap32(exact)
            assert C1[i, j] == _wrap32(exact + int(C0[i, j]))


def test_int32_oracle_small_values_match_float_oracle(oracle_mod):
    A, B = inputs.gemm_operands(17, 13, 29, seed=3, dist="integers")
    Ci = oracle_mod.gemm_i32(A.astype(np.int32), B.astype(np.int32))
    assert np.array_equal(Ci.astype(np.float64), oracle_mod.gemm(A, B))
