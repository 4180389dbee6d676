"""Parity of the FP32 SIMT family (paper-form, register-blocked, direct) with the
FP64 oracle, through the C ABI on the GPU."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_04348_gb300 import inputs, pgk

from helpers import assert_fp32_gemm

pytestmark = pytest.mark.gpu

GRID = [(b0, b1, s) for b0 in (8, 16, 32) for b1 in (8, 16, 32) for s in (1, 2, 4)]


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


@pytest.fixture(scope="module")
def machine(dev):
    return pgk.machine_query(0)


def _run(dev, A, B, prog=None, beta=0, C0=None, case=None):
    At = torch.from_numpy(A).to(dev)
    Bt = torch.from_numpy(B).to(dev)
    C = torch.from_numpy(C0).to(dev) if C0 is not None else torch.full(
        (A.shape[0], B.shape[1]), float("nan"), device=dev)
    if case is not None:
        pgk.gemm_case(case, At, Bt, C, beta=beta)
    else:
        pgk.gemm(At, Bt, C, pgk.F32, prog, beta=beta)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def test_machine_parameters(machine):
    assert machine.cc_major == 10 and machine.sm_count >= 100
    assert machine.max_threads_per_block == 1024 and machine.smem_per_block_optin >= 200 * 1024


def test_config1_every_feasible_point(dev, machine):
    """256^3, uniform[-1,1] seed 0, every (B0,B1,s) of {8,16,32}^2 x {1,2,4}."""
    A, B = inputs.gemm_operands(256, 256, 256, seed=0)
    feasible = 0
    for b0, b1, s in GRID:
        prog = pgk.params(b0, b1, s)
        st, c = pgk.select_case(machine, 256, 256, 256, pgk.F32, prog, raise_on_error=False)
        if b0 > b1 * s:
            assert st == 2
            continue
        assert st == 0 and c.leaf == pgk.LEAF_4A3A
        feasible += 1
        assert_fp32_gemm(_run(dev, A, B, prog), A, B)
    assert feasible == 23


def test_every_leaf_runs_on_the_gpu(dev, machine):
    """Leaves (3b,4a) and (3b,4b) are reached by shrinking Z_B in a copy of the
    real machine; the chosen variants then run on the real GPU."""
    A, B = inputs.gemm_operands(193, 177, 161, seed=3)
    seen = set()
    for b0, b1, s in GRID:
        if b0 > b1 * s:
            continue
        for zb in (machine.smem_per_block_optin, 4 * (b0 * b0 + b0 * b1 * s) - 4, 4 * (b0 * b0 + b0 * b1) - 4):
            m = pgk.Machine(*[getattr(machine, f) for f, _ in pgk.Machine._fields_])
            m.smem_per_block_optin = zb
            st, c = pgk.select_case(m, 193, 177, 161, pgk.F32, pgk.params(b0, b1, s), raise_on_error=False)
            assert st == 0
            seen.add(c.leaf)
            assert_fp32_gemm(_run(dev, A, B, case=c), A, B)
    assert seen == {0, 1, 2}


def _all_simt_params():
    out = []
    for i in range(pgk.num_variants()):
        v = pgk.variant_info_get(i)
        if v.family == pgk.FAM_RB:
            out.append(pgk.params(v.B0, v.B1, v.s, v.sr, v.tile))
    out += [pgk.params(16, 16, s) for s in (1, 2, 4, 8)] + [pgk.params(8, 32, 4, 1, 24)]
    return out


def test_integer_inputs_exact_every_variant(dev):
    """Integers in [-4,4] with K*16 < 2^24: every partial sum is exact in FP32,
    so each variant must agree with the oracle bit for bit."""
    A, B = inputs.gemm_operands(150, 130, 300, seed=5, dist="integers")
    ref = oracle.gemm(A, B)
    for prog in _all_simt_params():
        C = _run(dev, A, B, prog)
        assert np.array_equal(C.astype(np.float64), ref), prog.as_tuple()


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (7, 5, 3), (257, 129, 65), (1001, 333, 517), (64, 1, 999)])
def test_ragged_shapes_every_variant(dev, M, N, K):
    A, B = inputs.gemm_operands(M, N, K, seed=M + N + K)
    for prog in _all_simt_params():
        assert_fp32_gemm(_run(dev, A, B, prog), A, B)


def test_unaligned_leading_dimensions_and_beta(dev):
    """lda, ldb, ldc not multiples of 4 (scalar paths) and the accumulate form."""
    M, N, K = 131, 97, 75
    A, B = inputs.gemm_operands(M, N, K, seed=11)
    C0 = inputs.uniform((M, N), 12)
    Ap = torch.zeros(M, K + 3, device=dev)
    Ap[:, :K] = torch.from_numpy(A).to(dev)
    Bp = torch.zeros(K, N + 1, device=dev)
    Bp[:, :N] = torch.from_numpy(B).to(dev)
    for prog in [pgk.params(16, 16, 8, 8, 8), pgk.params(8, 16, 2), pgk.params(16, 8, 8, 8, 16)]:
        Cp = torch.zeros(M, N + 5, device=dev)
        Cp[:, :N] = torch.from_numpy(C0).to(dev)
        pgk.gemm(Ap, Bp, Cp, pgk.F32, prog, beta=1, M=M, N=N, K=K)
        torch.cuda.synchronize()
        assert_fp32_gemm(Cp[:, :N].cpu().numpy(), A, B, C0=C0, beta=1)
        assert torch.all(Cp[:, N:] == 0)


def test_register_predicate_matches_the_driver(dev):
    """The register-file counter predicts exactly the largest block the driver
    accepts for every compiled variant (cudaFuncAttributes.maxThreadsPerBlock)."""
    for i in range(pgk.num_variants()):
        v = pgk.variant_info_get(i)
        if v.family not in (pgk.FAM_PAPER, pgk.FAM_DIRECT):
            continue
        best = 0
        for threads in range(32, 1025, 32):
            alloc = (threads // 32) * ((v.regs * 32 + 255) // 256 * 256)
            if alloc <= 65536:
                best = threads
        assert best == v.max_threads, (v.family, v.s, v.regopt, v.regs, v.max_threads)


def test_launch_outcome_matches_prediction(dev, machine):
    """Predicted feasible <=> the launch does not fail (32 x 32 blocks)."""
    A, B = inputs.gemm_operands(64, 64, 64, seed=1)
    for s in (1, 2, 4, 8):
        st, c = pgk.select_case(machine, 64, 64, 64, pgk.F32, pgk.params(32, 32, s), raise_on_error=False)
        assert st == 0
        assert_fp32_gemm(_run(dev, A, B, case=c), A, B)


@pytest.mark.parametrize("M,N,K", [(8192, 8192, 8192), (4096, 4096, 4096), (8192, 1024, 4096),
                                   (16384, 64, 16384)])
def test_full_size_sampled_rows(dev, M, N, K):
    """The FP32 workload sizes (4096^3, 8192^3, 8192 x 1024 x 4096 and the skinny
    16384 x 64 x 16384) with the default (tuned-or-default) parameters; 24 sampled
    rows checked against the oracle row by row."""
    A, B = inputs.gemm_operands(M, N, K, seed=0)
    rows = np.unique(np.concatenate([[0, M - 1], np.random.default_rng(0).integers(0, M, 22)]))
    At = torch.from_numpy(A).to(dev)
    Bt = torch.from_numpy(B).to(dev)
    C = torch.empty(M, N, device=dev)
    pgk.gemm(At, Bt, C, pgk.F32, None)
    torch.cuda.synchronize()
    Cs = C[torch.from_numpy(rows).to(dev)].cpu().numpy()
    assert_fp32_gemm(Cs, A, B, rows=rows)


@pytest.mark.parametrize("M,N,K", [(64, 64, 8192), (100, 70, 5000), (256, 64, 16384)])
def test_split_k_exact_on_integers(dev, M, N, K):
    """Few output tiles and a long K take the split-K path (slices summed in
    order); integer-valued FP32 operands keep every partial sum exact, so the
    result must equal the oracle bit for bit, for every register-blocked variant."""
    A, B = inputs.gemm_operands(M, N, K, seed=K, dist="integers")
    ref = oracle.gemm(A, B)
    for prog in _all_simt_params():
        if prog.sr > 1:
            assert np.array_equal(_run(dev, A, B, prog).astype(np.float64), ref), prog.as_tuple()


@pytest.mark.parametrize("paired", [1, 0])
def test_fma_probe_below_the_derived_peak(dev, machine, paired):
    """The FFMA probe cannot beat SM count x 128 lanes x 2 flop x the maximum SM
    clock, and a dependency-free FMA stream should come close to it."""
    blocks, iters = machine.sm_count * 8, 4000
    sink = torch.empty(blocks * 256, device=dev)
    pgk.simt_peak_probe(blocks, iters, paired, sink)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    pgk.simt_peak_probe(blocks, iters, paired, sink)
    b.record()
    b.synchronize()
    tflops = blocks * 256 * iters * 16 * (2 if paired else 1) * 2 / a.elapsed_time(b) / 1e9
    peak = machine.sm_count * 128 * 2 * 2.1e9 / 1e12  # TFLOP/s; 2100 MHz bounds the 2070 MHz maximum
    assert 0.3 * peak < tflops < peak
    assert torch.isfinite(sink).all()
