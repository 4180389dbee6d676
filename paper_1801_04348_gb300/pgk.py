"""Thin ctypes binding of the C ABI in include/pgk.h (argument marshalling only).

Every function here forwards to the entry point of the same name in the
in-tree library `_build/libpgk.so`; all arithmetic runs in that library's CUDA
kernels.  Tensors are passed as raw device pointers (`tensor.data_ptr()`) and
streams as raw handles; nothing falls back to a CPU or PyTorch implementation:
if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpgk.so")

PGK_OK = 0
STATUS = {0: "PGK_OK", 1: "PGK_ERR_INVALID_ARG", 2: "PGK_ERR_INFEASIBLE", 3: "PGK_ERR_UNSUPPORTED",
          4: "PGK_ERR_ALIGNMENT", 5: "PGK_ERR_CUDA", 6: "PGK_ERR_TIMEOUT", 7: "PGK_ERR_NO_MEMORY"}
F32, BF16, FP8_E4M3, SPLIT_BF16, I32 = 0, 1, 2, 3, 4
DTYPES = {"f32": F32, "bf16": BF16, "fp8": FP8_E4M3, "split": SPLIT_BF16, "i32": I32}
LEAF_4A3A, LEAF_3B4A, LEAF_3B4B = 0, 1, 2
(FAM_PAPER, FAM_RB, FAM_DIRECT, FAM_TC_BF16, FAM_TC_SPLIT, FAM_TC_FP8, FAM_PAPER_I32, FAM_RB_I32,
 FAM_DIRECT_I32, FAM_TRANSPOSE, FAM_TRANSPOSE_DIRECT, FAM_JACOBI, FAM_JACOBI_DIRECT) = range(13)
STENCIL_REG_CLASSES = 5
REG_CLASSES = 11
MLP_PARAMS = 4737


class PgkError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class Machine(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in (
        "max_threads_per_block", "smem_per_block", "smem_per_block_optin", "regs_per_block",
        "regs_per_sm", "max_regs_per_thread", "max_threads_per_sm", "sm_count", "warp_size",
        "cc_major", "cc_minor", "l2_bytes")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("B0", "B1", "s", "sr", "tile")]

    def as_tuple(self):
        return (self.B0, self.B1, self.s, self.sr, self.tile)


class Case(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int), ("variant_id", ctypes.c_int), ("family", ctypes.c_int),
                ("regopt", ctypes.c_int), ("smem_bytes", ctypes.c_int), ("regs", ctypes.c_int),
                ("threads", ctypes.c_int), ("params", Params)]


class VariantInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in (
        "family", "s", "sr", "B0", "B1", "tile", "regopt", "regs", "max_threads")]


class Problem(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("N", ctypes.c_int), ("K", ctypes.c_int),
                ("lda", ctypes.c_int), ("ldb", ctypes.c_int), ("ldc", ctypes.c_int),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p)]


_i, _p, _f = ctypes.c_int, ctypes.c_void_p, ctypes.c_float
_SIGS = {
    "pgk_abi_version": (_i, []),
    "pgk_status_string": (ctypes.c_char_p, [_i]),
    "pgk_last_error": (ctypes.c_char_p, []),
    "pgk_machine_query": (_i, [_i, ctypes.POINTER(Machine)]),
    "pgk_num_variants": (_i, []),
    "pgk_variant_info_get": (_i, [_i, ctypes.POINTER(VariantInfo)]),
    "pgk_select_case": (_i, [ctypes.POINTER(Machine), _i, _i, _i, _i, ctypes.POINTER(Params),
                             ctypes.POINTER(Case)]),
    "pgk_select_case_regs": (_i, [ctypes.POINTER(Machine), ctypes.POINTER(ctypes.c_int), _i, _i, _i,
                                  _i, ctypes.POINTER(Params), ctypes.POINTER(Case)]),
    "pgk_gemm": (_i, [_i, _i, _i, _i, _p, _i, _p, _i, _p, _i, _i, ctypes.POINTER(Params), _p]),
    "pgk_gemm_i32": (_i, [_i, _i, _i, _p, _i, _p, _i, _p, _i, _i, ctypes.POINTER(Params), _p]),
    "pgk_gemm_case": (_i, [ctypes.POINTER(Case), _i, _i, _i, _p, _i, _p, _i, _p, _i, _i, _p]),
    "pgk_gemm_grouped": (_i, [_i, ctypes.POINTER(Problem), _i, ctypes.POINTER(Params), _i, _i, _p]),
    "pgk_select_case_transpose": (_i, [ctypes.POINTER(Machine), ctypes.POINTER(ctypes.c_int), _i, _i,
                                       ctypes.POINTER(Params), ctypes.POINTER(Case)]),
    "pgk_transpose": (_i, [_i, _i, _p, _i, _p, _i, ctypes.POINTER(Params), _p]),
    "pgk_transpose_case": (_i, [ctypes.POINTER(Case), _i, _i, _p, _i, _p, _i, _p]),
    "pgk_select_case_jacobi": (_i, [ctypes.POINTER(Machine), ctypes.POINTER(ctypes.c_int), _i,
                                    ctypes.POINTER(Params), ctypes.POINTER(Case)]),
    "pgk_jacobi": (_i, [_i, _i, _p, ctypes.POINTER(Params), _p]),
    "pgk_jacobi_case": (_i, [ctypes.POINTER(Case), _i, _i, _p, _p]),
    "pgk_cvt_bf16": (_i, [_i, _i, _p, _i, _p, _i, _i, _p]),
    "pgk_split_bf16": (_i, [_i, _i, _p, _i, _p, _p, _i, _i, _p]),
    "pgk_quant_fp8": (_i, [_i, _i, _p, _i, _p, _i, _p, _i, _i, _p]),
    "pgk_gemm_lowp": (_i, [_i, _i, _i, _i, _p, _i, _p, _i, _p, _p, _p, _p, _p, _i, _i,
                           ctypes.POINTER(Params), _p]),
    "pgk_gemm_host": (_i, [_i, _i, _i, _i, _p, _i, _p, _i, _p, _i, _i, ctypes.POINTER(Params), _p]),
    "pgk_relerr": (_i, [_i, _i, _p, _i, _p, _i, _p, _p, _p]),
    "pgk_simt_peak_probe": (_i, [_i, _i, _i, _p, _p]),
    "pgk_mlp_forward": (_i, [_i, _p, _p, _p, _p]),
    "pgk_mlp_loss_grad": (_i, [_i, _p, _p, _p, _p, _p, _p, _p]),
    "pgk_mlp_loss_grad_noalloc": (_i, [_i, _p, _p, _p, _p, _p, _p, _p]),
    "pgk_mlp_adam": (_i, [_i, _p, _p, _p, _p, _i, _f, _f, _f, _f, _p]),
    "pgk_autotune": (_i, [_i, _i, _i, _i, _p, _i, _p, _i, _p, _i, ctypes.POINTER(Params), _i, _i,
                          ctypes.POINTER(ctypes.c_float), ctypes.POINTER(Params), ctypes.c_char_p, _p]),
    "pgk_default_candidates": (_i, [_i, ctypes.POINTER(Params), _i]),
    "pgk_grouped_variants": (_i, [ctypes.POINTER(Params), _i, ctypes.POINTER(ctypes.c_int)]),
    "pgk_autotune_grouped": (_i, [_i, ctypes.POINTER(Problem), ctypes.POINTER(Params), _i, _i,
                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(Params), _p]),
    "pgk_costmodel_load": (_i, [_i, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                ctypes.POINTER(ctypes.c_float), _f, _f, _i]),
    "pgk_costmodel_clear": (_i, [_i]),
    "pgk_tune_cache_put": (_i, [_i, _i, _i, _i, ctypes.POINTER(Params)]),
    "pgk_tune_cache_get": (_i, [_i, _i, _i, _i, ctypes.POINTER(Params)]),
    "pgk_tune_cache_save": (_i, [ctypes.c_char_p]),
    "pgk_tune_cache_load": (_i, [ctypes.c_char_p]),
    "pgk_check_device_error": (_i, []),
    "pgk_selftest_bounded_wait": (_i, [ctypes.c_ulonglong, _p]),
    "pgk_shutdown": (_i, []),
}

_lib = None


def lib():
    """Load the library (raises if it was not built; there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libpgk.so not built at {LIB_PATH}: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def symbols():
    return list(_SIGS)


def last_error() -> str:
    return lib().pgk_last_error().decode()


def _check(status: int, fn: str):
    if status != PGK_OK:
        raise PgkError(status, fn, last_error())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def params(B0, B1, s, sr=1, tile=0) -> Params:
    return Params(B0, B1, s, sr, tile)


# ---------------------------------------------------------------- machine
def machine_query(device: int = 0) -> Machine:
    m = Machine()
    _check(lib().pgk_machine_query(device, ctypes.byref(m)), "pgk_machine_query")
    return m


def num_variants() -> int:
    return lib().pgk_num_variants()


def variant_info_get(i: int) -> VariantInfo:
    v = VariantInfo()
    _check(lib().pgk_variant_info_get(i, ctypes.byref(v)), "pgk_variant_info_get")
    return v


def select_case(machine: Machine, M, N, K, dtype, prog: Params, raise_on_error=True):
    c = Case()
    st = lib().pgk_select_case(ctypes.byref(machine), M, N, K, dtype, ctypes.byref(prog), ctypes.byref(c))
    if raise_on_error:
        _check(st, "pgk_select_case")
        return c
    return st, c


def select_case_regs(machine: Machine, regs, M, N, K, dtype, prog: Params):
    """Returns (status, Case) without raising (used for brute-force comparisons)."""
    arr = (ctypes.c_int * REG_CLASSES)(*regs)
    c = Case()
    st = lib().pgk_select_case_regs(ctypes.byref(machine), arr, M, N, K, dtype, ctypes.byref(prog),
                                    ctypes.byref(c))
    return st, c


# ------------------------------------------------------------------- GEMM
def gemm(A, B, C, dtype=F32, prog: Params | None = None, beta=0, stream=None, M=None, N=None,
         K=None, lda=None, ldb=None, ldc=None):
    M = A.shape[0] if M is None else M
    K = A.shape[1] if K is None else K
    N = B.shape[1] if N is None else N
    lda = A.stride(0) if lda is None else lda
    ldb = B.stride(0) if ldb is None else ldb
    ldc = C.stride(0) if ldc is None else ldc
    st = lib().pgk_gemm(M, N, K, dtype, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, int(beta),
                        ctypes.byref(prog) if prog is not None else None, _stream(stream))
    _check(st, "pgk_gemm")


def gemm_host(A, B, C, dtype=F32, prog: Params | None = None, beta=0, stream=None):
    """GEMM on host (CPU) FP32 tensors, pinned for full copy rate; asynchronous on
    `stream`: A and B must keep their values and C must not be read until the
    stream has completed the call."""
    M, K = A.shape
    N = B.shape[1]
    st = lib().pgk_gemm_host(M, N, K, dtype, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C),
                             C.stride(0), int(beta), ctypes.byref(prog) if prog is not None else None,
                             _stream(stream))
    _check(st, "pgk_gemm_host")


def gemm_i32(A, B, C, prog: Params | None = None, beta=0, stream=None):
    """int32 GEMM modulo 2^32 (torch.int32 device tensors)."""
    M, K = A.shape
    N = B.shape[1]
    st = lib().pgk_gemm_i32(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C), C.stride(0),
                            int(beta), ctypes.byref(prog) if prog is not None else None,
                            _stream(stream))
    _check(st, "pgk_gemm_i32")


def gemm_case(case: Case, A, B, C, beta=0, stream=None):
    M, K = A.shape
    N = B.shape[1]
    st = lib().pgk_gemm_case(ctypes.byref(case), M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0),
                             _ptr(C), C.stride(0), int(beta), _stream(stream))
    _check(st, "pgk_gemm_case")


def make_problems(triples):
    """triples: list of (A, B, C) device tensors -> ctypes array of Problem."""
    arr = (Problem * len(triples))()
    for i, (A, B, C) in enumerate(triples):
        arr[i] = Problem(A.shape[0], B.shape[1], A.shape[1], A.stride(0), B.stride(0), C.stride(0),
                         _ptr(A), _ptr(B), _ptr(C))
    return arr


def gemm_grouped(problems, dtype=F32, prog: Params | None = None, use_graph=0, beta=0, stream=None):
    st = lib().pgk_gemm_grouped(len(problems), problems, dtype,
                                ctypes.byref(prog) if prog is not None else None, int(use_graph),
                                int(beta), _stream(stream))
    _check(st, "pgk_gemm_grouped")


def grouped_variants() -> list:
    n = ctypes.c_int(0)
    lib().pgk_grouped_variants(None, 0, ctypes.byref(n))
    arr = (Params * n.value)()
    lib().pgk_grouped_variants(arr, n.value, None)
    return [arr[i] for i in range(n.value)]


def autotune_grouped(problems, candidates=None, reps=3, stream=None):
    """Returns (best Params, list of (Params, ms))."""
    cand = candidates if candidates is not None else grouped_variants()
    arr = (Params * len(cand))(*cand)
    ms = (ctypes.c_float * len(cand))()
    best = Params()
    _check(lib().pgk_autotune_grouped(len(problems), problems, arr, len(cand), reps, ms,
                                      ctypes.byref(best), _stream(stream)), "pgk_autotune_grouped")
    return best, [(cand[i], ms[i]) for i in range(len(cand))]


# ------------------------------------------- transposition and 1D Jacobi
def select_case_transpose(machine: Machine, rows, cols, prog: Params, regs=None):
    """Returns (status, Case); regs = 5 register counts or None (query the GPU)."""
    arr = (ctypes.c_int * STENCIL_REG_CLASSES)(*regs) if regs is not None else None
    c = Case()
    st = lib().pgk_select_case_transpose(ctypes.byref(machine), arr, rows, cols, ctypes.byref(prog),
                                         ctypes.byref(c))
    return st, c


def transpose(src, dst, prog: Params | None = None, stream=None):
    rows, cols = src.shape
    _check(lib().pgk_transpose(rows, cols, _ptr(src), src.stride(0), _ptr(dst), dst.stride(0),
                               ctypes.byref(prog) if prog is not None else None, _stream(stream)),
           "pgk_transpose")


def transpose_case(case: Case, src, dst, stream=None):
    rows, cols = src.shape
    _check(lib().pgk_transpose_case(ctypes.byref(case), rows, cols, _ptr(src), src.stride(0), _ptr(dst),
                                    dst.stride(0), _stream(stream)), "pgk_transpose_case")


def select_case_jacobi(machine: Machine, n, prog: Params, regs=None):
    arr = (ctypes.c_int * STENCIL_REG_CLASSES)(*regs) if regs is not None else None
    c = Case()
    st = lib().pgk_select_case_jacobi(ctypes.byref(machine), arr, n, ctypes.byref(prog), ctypes.byref(c))
    return st, c


def jacobi(a, n, steps, prog: Params | None = None, stream=None):
    """a: int32 device tensor of 2n entries, updated in place."""
    _check(lib().pgk_jacobi(n, steps, _ptr(a), ctypes.byref(prog) if prog is not None else None,
                            _stream(stream)), "pgk_jacobi")


def jacobi_case(case: Case, a, n, steps, stream=None):
    _check(lib().pgk_jacobi_case(ctypes.byref(case), n, steps, _ptr(a), _stream(stream)),
           "pgk_jacobi_case")


# --------------------------------------------------------- low precision
def cvt_bf16(src, dst, transpose=0, stream=None, rows=None, cols=None):
    rows = src.shape[0] if rows is None else rows
    cols = src.shape[1] if cols is None else cols
    _check(lib().pgk_cvt_bf16(rows, cols, _ptr(src), src.stride(0), _ptr(dst), dst.stride(0),
                              int(transpose), _stream(stream)), "pgk_cvt_bf16")


def split_bf16(src, hi, lo, transpose=0, stream=None):
    rows, cols = src.shape
    _check(lib().pgk_split_bf16(rows, cols, _ptr(src), src.stride(0), _ptr(hi), _ptr(lo), hi.stride(0),
                                int(transpose), _stream(stream)), "pgk_split_bf16")


def quant_fp8(src, dst, scales, transpose=0, stream=None):
    rows, cols = src.shape
    _check(lib().pgk_quant_fp8(rows, cols, _ptr(src), src.stride(0), _ptr(dst), dst.stride(0),
                               _ptr(scales), scales.stride(0), int(transpose), _stream(stream)),
           "pgk_quant_fp8")


def gemm_lowp(M, N, K, dtype, A, lda, Bt, ldbt, C, ldc, A_lo=None, Bt_lo=None, scaleA=None,
              scaleB=None, beta=0, prog: Params | None = None, stream=None):
    _check(lib().pgk_gemm_lowp(M, N, K, dtype, _ptr(A), lda, _ptr(Bt), ldbt, _ptr(A_lo), _ptr(Bt_lo),
                               _ptr(scaleA), _ptr(scaleB), _ptr(C), ldc, int(beta),
                               ctypes.byref(prog) if prog is not None else None, _stream(stream)),
           "pgk_gemm_lowp")


# ------------------------------------------------------ error measurement
def relerr(C, Cref, out, row_index=None, stream=None, rows=None, cols=None):
    rows = Cref.shape[0] if rows is None else rows
    cols = Cref.shape[1] if cols is None else cols
    _check(lib().pgk_relerr(rows, cols, _ptr(C), C.stride(0), _ptr(Cref), Cref.stride(0),
                            _ptr(row_index), _ptr(out), _stream(stream)), "pgk_relerr")


def simt_peak_probe(blocks, iters, paired, sink, stream=None):
    """FP32 FMA throughput probe; flops = blocks * 256 * iters * 16 * (2 if paired else 1) * 2."""
    _check(lib().pgk_simt_peak_probe(int(blocks), int(iters), int(paired), _ptr(sink), _stream(stream)),
           "pgk_simt_peak_probe")


# ------------------------------------------------------------- cost model
def mlp_forward(X, theta, y, stream=None):
    _check(lib().pgk_mlp_forward(X.shape[0], _ptr(X), _ptr(theta), _ptr(y), _stream(stream)),
           "pgk_mlp_forward")


def mlp_loss_grad(X, t, theta, grad, loss, idx=None, stream=None, n=None):
    n = (idx.shape[0] if idx is not None else X.shape[0]) if n is None else n
    _check(lib().pgk_mlp_loss_grad(n, _ptr(idx), _ptr(X), _ptr(t), _ptr(theta), _ptr(grad), _ptr(loss),
                                   _stream(stream)), "pgk_mlp_loss_grad")


def mlp_loss_grad_noalloc(X, t, theta, grad, loss, idx=None, stream=None, n=None):
    """pgk_mlp_loss_grad_noalloc: the gradient without any device allocation
    (static scratch, at most 2048 samples per call)."""
    n = (idx.shape[0] if idx is not None else X.shape[0]) if n is None else n
    _check(lib().pgk_mlp_loss_grad_noalloc(n, _ptr(idx), _ptr(X), _ptr(t), _ptr(theta), _ptr(grad),
                                           _ptr(loss), _stream(stream)), "pgk_mlp_loss_grad_noalloc")


def mlp_adam(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().pgk_mlp_adam(theta.numel(), _ptr(theta), _ptr(grad), _ptr(m), _ptr(v), int(step),
                              lr, beta1, beta2, eps, _stream(stream)), "pgk_mlp_adam")


# --------------------------------------------------------------- autotune
def default_candidates(dtype) -> list:
    n = lib().pgk_default_candidates(dtype, None, 0)
    arr = (Params * n)()
    lib().pgk_default_candidates(dtype, arr, n)
    return [arr[i] for i in range(n)]


def autotune(A, B, C, dtype=F32, candidates=None, reps=3, log_path=None, stream=None):
    """Returns (best Params, list of (Params, ms))."""
    M, K = A.shape
    N = B.shape[1]
    cand = candidates if candidates is not None else default_candidates(dtype)
    arr = (Params * len(cand))(*cand)
    ms = (ctypes.c_float * len(cand))()
    best = Params()
    st = lib().pgk_autotune(M, N, K, dtype, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C),
                            C.stride(0), arr, len(cand), reps, ms, ctypes.byref(best),
                            log_path.encode() if log_path else None, _stream(stream))
    _check(st, "pgk_autotune")
    return best, [(cand[i], ms[i]) for i in range(len(cand))]


def costmodel_load(dtype, theta, mu, sd, tmu, tsd, k=3):
    """Installs a trained cost model (host arrays) for pgk_gemm's learned selection."""
    th = (ctypes.c_float * len(theta))(*[float(x) for x in theta])
    m = (ctypes.c_float * 7)(*[float(x) for x in mu])
    s = (ctypes.c_float * 7)(*[float(x) for x in sd])
    _check(lib().pgk_costmodel_load(dtype, th, m, s, float(tmu), float(tsd), int(k)),
           "pgk_costmodel_load")


def costmodel_load_file(dtype, path, k=3):
    import json
    with open(path) as f:
        d = json.load(f)
    costmodel_load(dtype, d["theta"], d["mu"], d["sd"], d["tmu"], d["tsd"], k)


def costmodel_clear(dtype):
    _check(lib().pgk_costmodel_clear(dtype), "pgk_costmodel_clear")


def tune_cache_put(M, N, K, dtype, p: Params):
    _check(lib().pgk_tune_cache_put(M, N, K, dtype, ctypes.byref(p)), "pgk_tune_cache_put")


def tune_cache_get(M, N, K, dtype):
    p = Params()
    st = lib().pgk_tune_cache_get(M, N, K, dtype, ctypes.byref(p))
    return p if st == PGK_OK else None


def tune_cache_save(path: str):
    _check(lib().pgk_tune_cache_save(path.encode()), "pgk_tune_cache_save")


def tune_cache_load(path: str):
    _check(lib().pgk_tune_cache_load(path.encode()), "pgk_tune_cache_load")


def check_device_error():
    _check(lib().pgk_check_device_error(), "pgk_check_device_error")


def selftest_bounded_wait(limit_ns=50_000_000, stream=None):
    _check(lib().pgk_selftest_bounded_wait(int(limit_ns), _stream(stream)), "pgk_selftest_bounded_wait")


def shutdown():
    _check(lib().pgk_shutdown(), "pgk_shutdown")
