"""Shared helpers for the GPU parity tests (host-side comparisons only)."""
import numpy as np

import oracle

U32 = 2.0 ** -24


def gamma(K, u=U32):
    return K * u / (1.0 - K * u)


def assert_fp32_gemm(C, A, B, C0=None, beta=0, rows=None, rel_tol=1e-5):
    """Element-wise forward-error bound |C - Cref| <= gamma_K (|A||B| + |C0|)
    (Higham's standard bound for a length-K FP32 dot product, with one more
    rounding for the beta term) and the relative Frobenius tolerance."""
    K = A.shape[1]
    ref = oracle.gemm(A, B, C0=C0, beta=float(beta), rows=rows)
    Ar = A if rows is None else A[rows]
    absAB = np.abs(Ar).astype(np.float64) @ np.abs(B).astype(np.float64)
    if beta:
        absAB = absAB + np.abs(C0 if rows is None else C0[rows]).astype(np.float64)
    Cg = np.asarray(C, dtype=np.float64)
    bound = gamma(K + (1 if beta else 0)) * absAB * 1.0001 + 1e-30
    bad = np.abs(Cg - ref) > bound
    assert not bad.any(), f"{bad.sum()} entries exceed the FP32 error bound"
    err = oracle.rel_frobenius(Cg, ref)
    assert err <= rel_tol, err
    return err
