"""Exhaustive tiny shapes: every M, N, K in [1, 9] through every compiled variant
of every form, against the long-double textbook product (element-wise bounds) and,
on small-integer inputs, bit for bit.  These sizes leave every tile ragged in all
three dimensions, so they exercise the zero-fill of the tails and the bounds of
the epilogue stores (Fig. "cudamul" guards only the p, q bounds; the kernels here
take arbitrary M, N, K >= 1)."""
import itertools

import numpy as np
import pytest
import torch

import oracle
from oracle import quant
from paper_1801_04348_gb300 import inputs, pgk

from helpers import gamma

pytestmark = pytest.mark.gpu

SIZES = list(itertools.product(range(1, 10), repeat=3))
TC_VARIANTS = {pgk.BF16: [(128, 256, 4), (128, 128, 6), (128, 256, 3), (128, 128, 4), (256, 256, 6)],
               pgk.SPLIT_BF16: [(128, 128, 3), (128, 256, 2), (128, 256, 4), (128, 128, 6),
                                (256, 256, 3), (256, 256, 6)],
               pgk.FP8_E4M3: [(128, 128, 6), (128, 256, 4)]}


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _simt_params():
    """Every register-blocked variant, the paper-form granularities and a
    direct-leaf-sized paper block."""
    out = []
    for i in range(pgk.num_variants()):
        v = pgk.variant_info_get(i)
        if v.family == pgk.FAM_RB:
            out.append(pgk.params(v.B0, v.B1, v.s, v.sr, v.tile))
    return out + [pgk.params(16, 16, s) for s in (1, 2, 4, 8)] + [pgk.params(8, 32, 4, 1, 24)]


def _t(x, dev):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def _simt_all(dev, A, B, progs):
    """C of every program, all launched before one synchronisation."""
    At, Bt = _t(A, dev), _t(B, dev)
    Cs = []
    for prog in progs:
        C = torch.full((A.shape[0], B.shape[1]), float("nan"), device=dev)
        pgk.gemm(At, Bt, C, pgk.F32, prog)
        Cs.append(C)
    torch.cuda.synchronize()
    return [C.cpu().numpy().astype(np.float64) for C in Cs]


def _prep(dev, A, B, form):
    """Prepared operands through the library's preparation entry points
    (K padded to 16 elements, B transposed)."""
    M, K = A.shape
    N = B.shape[1]
    Kp = (K + 15) // 16 * 16
    At, Bt = _t(A, dev), _t(B, dev)
    if form == pgk.FP8_E4M3:
        a = torch.zeros(M, Kp, dtype=torch.uint8, device=dev)
        b = torch.zeros(N, Kp, dtype=torch.uint8, device=dev)
        sa = torch.zeros(1, 1, device=dev)
        sb = torch.zeros(1, 1, device=dev)
        pgk.quant_fp8(At, a, sa, 0)
        pgk.quant_fp8(Bt, b, sb, 1)
        return dict(A=a, Bt=b, scaleA=sa, scaleB=sb)
    a = torch.zeros(M, Kp, dtype=torch.int16, device=dev)
    b = torch.zeros(N, Kp, dtype=torch.int16, device=dev)
    if form == pgk.BF16:
        pgk.cvt_bf16(At, a, 0)
        pgk.cvt_bf16(Bt, b, 1)
        return dict(A=a, Bt=b)
    al, bl = torch.zeros_like(a), torch.zeros_like(b)
    pgk.split_bf16(At, a, al, 0)
    pgk.split_bf16(Bt, b, bl, 1)
    return dict(A=a, Bt=b, A_lo=al, Bt_lo=bl)


def _tc_all(dev, A, B, form):
    """C of every compiled tile program of `form` on prepared operands, plus the
    library-prepared call (pgk_gemm on FP32 inputs, tuned program) last."""
    M, K = A.shape
    N = B.shape[1]
    ops = _prep(dev, A, B, form)
    Kp = ops["A"].stride(0)
    Cs = []
    for bm, bn, st in TC_VARIANTS[form]:
        C = torch.full((M, N), float("nan"), device=dev)
        pgk.gemm_lowp(M, N, K, form, ops["A"], Kp, ops["Bt"], Kp, C, N, A_lo=ops.get("A_lo"),
                      Bt_lo=ops.get("Bt_lo"), scaleA=ops.get("scaleA"),
                      scaleB=ops.get("scaleB"), prog=pgk.params(bm, bn, st, 0, 0))
        Cs.append(C)
    C = torch.full((M, N), float("nan"), device=dev)
    pgk.gemm(_t(A, dev), _t(B, dev), C, form, None)
    Cs.append(C)
    torch.cuda.synchronize()
    pgk.check_device_error()
    return [C.cpu().numpy().astype(np.float64) for C in Cs]


def _dequantised_reference(A, B, form):
    """The long-double product of the operands the tensor cores see: the BF16
    roundings, the three split products, or the dequantised FP8 codes."""
    ld = oracle.gemm_longdouble
    f = lambda x: x.astype(np.float64)
    if form == pgk.BF16:
        return ld(f(quant.bf16_rn(A)), f(quant.bf16_rn(B)))
    if form == pgk.SPLIT_BF16:
        ha, la = quant.split_bf16(A)
        hb, lb = quant.split_bf16(B)
        return ld(f(ha), f(hb)) + ld(f(ha), f(lb)) + ld(f(la), f(hb))
    ca, sa = quant.fp8_tile_quant(A)
    cb, sb = quant.fp8_tile_quant(B)
    return ld(quant.fp8_dequant(ca, sa), quant.fp8_dequant(cb, sb))


def test_simt_every_tiny_shape_within_the_fp32_bound(dev):
    """Uniform[-1,1] inputs: |C - C_ld| <= gamma_K (|A||B|) element by element
    for every SIMT program at every shape in [1, 9]^3."""
    progs = _simt_params()
    for M, N, K in SIZES:
        A, B = inputs.gemm_operands(M, N, K, seed=100 * M + 10 * N + K)
        ref = oracle.gemm_longdouble(A, B)
        bound = gamma(K) * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)) + 1e-30
        for prog, C in zip(progs, _simt_all(dev, A, B, progs)):
            assert np.all(np.abs(C - ref) <= bound), ((M, N, K), prog.as_tuple())


def test_simt_every_tiny_shape_exact_on_integers_and_zeros(dev):
    """Small integers: every partial sum is exact in FP32, so every program equals
    the long-double product bit for bit; an all-zero A gives an all-zero C and a
    rank-one pair (outer products of integer vectors) its closed form."""
    progs = _simt_params()
    for M, N, K in SIZES:
        A = inputs.integers((M, K), 3 * M + K, -4, 4)
        B = inputs.integers((K, N), 5 * N + K, -4, 4)
        ref = oracle.gemm_longdouble(A, B)
        for prog, C in zip(progs, _simt_all(dev, A, B, progs)):
            assert np.array_equal(C, ref), ((M, N, K), prog.as_tuple())
    for M, N, K in [(9, 7, 5), (1, 9, 9), (8, 8, 8)]:
        Z = np.zeros((M, K), np.float32)
        x = inputs.integers((M, 1), 1, -3, 3)
        y = inputs.integers((1, K), 2, -3, 3)
        z = inputs.integers((K, 1), 3, -3, 3)
        w = inputs.integers((1, N), 4, -3, 3)
        B = z @ w
        rank1 = (x @ y).astype(np.float32)
        closed = float((y @ z)[0, 0]) * (x.astype(np.float64) @ w.astype(np.float64))
        for prog, C in zip(progs, _simt_all(dev, Z, B, progs)):
            assert np.array_equal(C, np.zeros((M, N))), prog.as_tuple()
        for prog, C in zip(progs, _simt_all(dev, rank1, B.astype(np.float32), progs)):
            assert np.array_equal(C, closed), prog.as_tuple()


@pytest.mark.parametrize("form", [pgk.BF16, pgk.SPLIT_BF16, pgk.FP8_E4M3])
def test_tensor_core_every_tiny_shape(dev, form):
    """Every tile program of the form (and the library-prepared call) at every
    shape in [1, 9]^3: within FP32 accumulation error of the long-double product
    of the operands the MMA sees, and bit for bit on small integers (FP8: a 7 in
    the single tile makes the scale 7 / 448 = 2^-6, so the codes are exact)."""
    for M, N, K in SIZES:
        A, B = inputs.gemm_operands(M, N, K, seed=100 * M + 10 * N + K + 7, dist="normal")
        ref = _dequantised_reference(A, B, form)
        k_eff = 3 * K if form == pgk.SPLIT_BF16 else K
        bound = (k_eff + 2) * 2.0 ** -24 * 2.5 * (
            np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)) + 1e-30
        for i, C in enumerate(_tc_all(dev, A, B, form)):
            assert np.all(np.abs(C - ref) <= bound), ((M, N, K), i)

        lo, hi = (-7, 7) if form == pgk.FP8_E4M3 else (-8, 8)
        A = inputs.integers((M, K), 3 * M + K, lo, hi)
        B = inputs.integers((K, N), 5 * N + K, lo, hi)
        if form == pgk.FP8_E4M3:
            A[0, 0] = 7
            B[0, 0] = 7
        ref = oracle.gemm_longdouble(A, B)
        for i, C in enumerate(_tc_all(dev, A, B, form)):
            assert np.array_equal(C, ref), ((M, N, K), i)
