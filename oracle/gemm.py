"""FP64 GEMM oracle (definition C = beta*C0 + A*B) -- TEST INFRASTRUCTURE ONLY.

Follows the product computed by the paper's blocked loop nest (Fig. "metamul",
Section 2) and its generated kernel (Fig. "cudamul"): every output coefficient
c[p][q] accumulates a[p][z]*b[z][q] over z.  Here that is the unblocked
definition, evaluated in binary64 by `pgk_oracle.c` (plain C, i-k-j loop, OpenMP
over rows).  Nothing in the product imports this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pgk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, dp, fp = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
        for name in ("oracle_gemm_f32in", "oracle_gemm_f64in"):
            fn = getattr(lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = [i64, i64, i64, fp, i64, fp, i64, ctypes.c_double, dp, i64,
                           dp, i64, dp, i64, ctypes.c_int]
        lib.oracle_gemm_longdouble.restype = ctypes.c_int
        lib.oracle_gemm_longdouble.argtypes = [i64, i64, i64, dp, dp, dp]
        lib.oracle_gemm_i32_wrap.restype = ctypes.c_int
        lib.oracle_gemm_i32_wrap.argtypes = [i64, i64, i64, fp, i64, fp, i64, ctypes.c_int, dp, i64,
                                             dp, i64]
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_max_threads.argtypes = []
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def gemm(A: np.ndarray, B: np.ndarray, C0: np.ndarray | None = None, beta: float = 0.0,
         rows: np.ndarray | None = None, nthreads: int = 0) -> np.ndarray:
    """Return beta*C0 + A@B in binary64 for the selected output rows.

    A (M x K) and B (K x N) are row-major arrays of float32 or float64; float32
    operands are promoted exactly.  `rows` selects output rows (all by default);
    the result has one row per selected row.  C0 is read only when beta != 0.
    """
    if A.ndim != 2 or B.ndim != 2 or A.shape[1] != B.shape[0]:
        raise ValueError("shape mismatch")
    M, K = A.shape
    N = B.shape[1]
    if A.dtype == np.float32 and B.dtype == np.float32:
        fn = _load().oracle_gemm_f32in
        A = np.ascontiguousarray(A)
        B = np.ascontiguousarray(B)
    else:
        fn = _load().oracle_gemm_f64in
        A = np.ascontiguousarray(A, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
    if rows is None:
        rows_arr = None
        nrows = M
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int64)
        if rows_arr.size and (rows_arr.min() < 0 or rows_arr.max() >= M):
            raise ValueError("row index out of range")
        nrows = rows_arr.size
    if beta != 0.0:
        if C0 is None or C0.shape != (M, N):
            raise ValueError("C0 must be M x N when beta != 0")
        C0 = np.ascontiguousarray(C0, dtype=np.float64)
    C = np.empty((nrows, N), dtype=np.float64)
    rc = fn(M, N, K, _ptr(A), K, _ptr(B), N, float(beta),
            _ptr(C0) if beta != 0.0 else None, N,
            _ptr(rows_arr) if rows_arr is not None else None, nrows,
            _ptr(C), N, int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle_gemm failed")
    return C


def gemm_longdouble(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Textbook i-j-k dot products in long double (self-check on tiny inputs)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[1]
    C = np.empty((M, N), dtype=np.float64)
    _load().oracle_gemm_longdouble(M, N, K, _ptr(A), _ptr(B), _ptr(C))
    return C


def gemm_i32(A: np.ndarray, B: np.ndarray, C0: np.ndarray | None = None,
             beta: int = 0) -> np.ndarray:
    """int32 C = beta*C0 + A@B modulo 2^32 (two's complement), the paper's data
    type; A (M x K), B (K x N) int32 row-major."""
    A = np.ascontiguousarray(A, dtype=np.int32)
    B = np.ascontiguousarray(B, dtype=np.int32)
    if A.shape[1] != B.shape[0]:
        raise ValueError("shape mismatch")
    M, K = A.shape
    N = B.shape[1]
    if beta:
        C0 = np.ascontiguousarray(C0, dtype=np.int32)
    C = np.empty((M, N), dtype=np.int32)
    rc = _load().oracle_gemm_i32_wrap(M, N, K, _ptr(A), K, _ptr(B), N, int(bool(beta)),
                                      _ptr(C0) if beta else None, N, _ptr(C), N)
    if rc != 0:
        raise RuntimeError("oracle_gemm_i32_wrap failed")
    return C


def rel_frobenius(C: np.ndarray, Cref: np.ndarray) -> float:
    """||C - Cref||_F / ||Cref||_F evaluated in binary64 (the error measure the
    tolerances are stated in)."""
    C = np.asarray(C, dtype=np.float64)
    Cref = np.asarray(Cref, dtype=np.float64)
    num = float(np.sum((C - Cref) ** 2))
    den = float(np.sum(Cref ** 2))
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return (num / den) ** 0.5
