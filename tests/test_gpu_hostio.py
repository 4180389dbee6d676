"""pgk_gemm_host: GEMM on host buffers (pinned and pageable), against the same
kernels on device buffers (bit for bit) and against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_04348_gb300 import inputs, pgk

from helpers import assert_fp32_gemm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _device_result(dev, A, B, dtype, prog, C0=None, beta=0):
    Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    C = torch.from_numpy(C0).to(dev) if C0 is not None else torch.empty(A.shape[0], B.shape[1], device=dev)
    pgk.gemm(Ad, Bd, C, dtype, prog, beta=beta)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def _host(x, pinned):
    t = torch.from_numpy(np.ascontiguousarray(x))
    return t.pin_memory() if pinned else t.clone()


FORMS = [(pgk.F32, pgk.params(16, 16, 8, 8, 8)), (pgk.SPLIT_BF16, pgk.params(128, 256, 2, 0, 0)),
         (pgk.BF16, pgk.params(128, 256, 4, 0, 0)), (pgk.FP8_E4M3, pgk.params(128, 256, 4, 0, 0)),
         (pgk.SPLIT_BF16, pgk.params(256, 256, 3, 0, 0)), (pgk.BF16, pgk.params(256, 256, 6, 0, 0))]


@pytest.mark.parametrize("dtype,prog", FORMS)
@pytest.mark.parametrize("pinned_c", [True, False])
def test_equals_device_path(dev, dtype, prog, pinned_c):
    """Two row panels split at row 256 (a multiple of the 128-row tiles, of the
    256-row CTA-pair tiles and of the FP8 scale blocks) give the whole-matrix result
    bit for bit."""
    M, N, K = 300, 272, 384
    A, B = inputs.gemm_operands(M, N, K, seed=3)
    Ah, Bh = _host(A, True), _host(B, True)
    Ch = _host(np.full((M, N), np.nan, np.float32), pinned_c)
    pgk.gemm_host(Ah, Bh, Ch, dtype, prog)
    torch.cuda.synchronize()
    assert np.array_equal(Ch.numpy(), _device_result(dev, A, B, dtype, prog))
    if dtype == pgk.F32:
        assert_fp32_gemm(Ch.numpy(), A, B)


@pytest.mark.parametrize("pinned_c", [True, False])
def test_beta_and_strided_host_views(dev, pinned_c):
    M, N, K = 257, 144, 200
    A, B = inputs.gemm_operands(M, N, K, seed=5)
    C0 = inputs.uniform((M, N), 9)
    prog = pgk.params(16, 16, 8, 8, 8)
    # views with leading dimensions larger than the rows
    Aw = torch.zeros(M, K + 24).pin_memory()
    Aw[:, :K] = torch.from_numpy(A)
    Bw = torch.zeros(K, N + 16).pin_memory()
    Bw[:, :N] = torch.from_numpy(B)
    Cw = torch.zeros(M, N + 8)
    Cw = Cw.pin_memory() if pinned_c else Cw
    Cw[:, :N] = torch.from_numpy(C0)
    pgk.gemm_host(Aw[:, :K], Bw[:, :N], Cw[:, :N], pgk.F32, prog, beta=1)
    torch.cuda.synchronize()
    got = Cw[:, :N].numpy()
    assert np.array_equal(got, _device_result(dev, A, B, pgk.F32, prog, C0=C0, beta=1))
    assert_fp32_gemm(got, A, B, C0=C0, beta=1)
    assert (Cw[:, N:].numpy() == 0).all()


def test_consecutive_calls_alternate_and_grow(dev):
    """Back-to-back calls without synchronisation (the input copies of one call
    overlap the previous GEMM), then a larger call that grows the buffer sets."""
    prog = pgk.params(16, 16, 8, 8, 8)
    shapes = [(256, 256, 256)] * 4 + [(512, 384, 640)]
    outs = []
    for i, (M, N, K) in enumerate(shapes):
        A, B = inputs.gemm_operands(M, N, K, seed=20 + i)
        Ah, Bh = _host(A, True), _host(B, True)
        Ch = _host(np.zeros((M, N), np.float32), True)
        pgk.gemm_host(Ah, Bh, Ch, pgk.F32, prog)
        outs.append((A, B, Ah, Bh, Ch))
    torch.cuda.synchronize()
    for A, B, _, _, Ch in outs:
        assert np.array_equal(Ch.numpy(), _device_result(dev, A, B, pgk.F32, prog))


@pytest.mark.parametrize("prog", [(128, 256, 2), (256, 256, 3)])
def test_sampled_rows_at_8192(dev, prog):
    """The split form at 8192^3 on pinned host buffers (single-CTA tiles: four panels
    of 19, 19, 19 and 7 tile rows; CTA pairs: 19 and 13 pair rows), rows on both sides
    of every panel boundary against the oracle."""
    M = N = K = 8192
    A, B = inputs.gemm_operands(M, N, K, seed=0, dist="normal")
    Ah, Bh = _host(A, True), _host(B, True)
    Ch = torch.empty(M, N).pin_memory()
    pgk.gemm_host(Ah, Bh, Ch, pgk.SPLIT_BF16, pgk.params(*prog, 0, 0))
    torch.cuda.synchronize()
    edges = [2431, 2432, 4863, 4864, 7295, 7296]
    rows = np.unique(np.concatenate([np.linspace(0, M - 1, 16).astype(np.int64), edges]))
    err = oracle.rel_frobenius(Ch.numpy()[rows].astype(np.float64), oracle.gemm(A, B, rows=rows))
    assert err <= 2e-5, err


def test_device_pointers_are_rejected(dev):
    A = torch.zeros(16, 16, device=dev)
    Bh = torch.zeros(16, 16).pin_memory()
    with pytest.raises(pgk.PgkError) as e:
        pgk.gemm_host(A, Bh, Bh.clone(), pgk.F32)
    assert e.value.status == 1  # PGK_ERR_INVALID_ARG


def test_pageable_inputs(dev):
    """Pageable (not pinned) A, B and C go through the driver's staged copies and give
    the same result."""
    M, N, K = 384, 200, 257
    A, B = inputs.gemm_operands(M, N, K, seed=31)
    prog = pgk.params(16, 16, 8, 8, 8)
    Ah, Bh = _host(A, False), _host(B, False)
    Ch = _host(np.zeros((M, N), np.float32), False)
    pgk.gemm_host(Ah, Bh, Ch, pgk.F32, prog)
    torch.cuda.synchronize()
    assert np.array_equal(Ch.numpy(), _device_result(dev, A, B, pgk.F32, prog))


def test_tuned_program_runs_every_panel(dev):
    """prog = NULL with a program in the tune cache for the whole shape: the panels
    are planned for it (256-row CTA-pair tiles here) and each runs it, so the
    result equals pgk_gemm's on the whole matrix, which runs the same program."""
    M, N, K = 1000, 520, 384
    A, B = inputs.gemm_operands(M, N, K, seed=13)
    pgk.tune_cache_put(M, N, K, pgk.SPLIT_BF16, pgk.params(256, 256, 3, 0, 0))
    Ah, Bh = _host(A, True), _host(B, True)
    Ch = _host(np.full((M, N), np.nan, np.float32), True)
    pgk.gemm_host(Ah, Bh, Ch, pgk.SPLIT_BF16, None)
    torch.cuda.synchronize()
    ref = _device_result(dev, A, B, pgk.SPLIT_BF16, None)
    assert np.array_equal(Ch.numpy(), ref)
    assert np.array_equal(ref, _device_result(dev, A, B, pgk.SPLIT_BF16, pgk.params(256, 256, 3, 0, 0)))


@pytest.mark.parametrize("dtype", [pgk.SPLIT_BF16, pgk.BF16])
def test_skinny_host_buffers_take_the_fused_program(dev, dtype):
    """N <= 64 on host buffers: with the fused-conversion program on one K slice
    every row panel reads its A in FP32 (B converted once) and the result equals
    the device path with the same program bit for bit; without parameters each
    panel selects it (with K slices where its row tiles leave SMs idle) and meets
    the form's tolerance against the FP64 oracle."""
    M, N, K = 1100, 64, 2048
    A, B = inputs.gemm_operands(M, N, K, seed=31)
    Ah, Bh = _host(A, True), _host(B, True)
    Ch = _host(np.full((M, N), np.nan, np.float32), True)
    fused = pgk.params(128, 64, 3 if dtype == pgk.SPLIT_BF16 else 4, 1, 0)   # one K slice
    pgk.gemm_host(Ah, Bh, Ch, dtype, fused)
    torch.cuda.synchronize()
    assert np.array_equal(Ch.numpy(), _device_result(dev, A, B, dtype, fused))
    Cn = _host(np.full((M, N), np.nan, np.float32), True)
    pgk.gemm_host(Ah, Bh, Cn, dtype, None)
    torch.cuda.synchronize()
    err = oracle.rel_frobenius(Cn.numpy().astype(np.float64), oracle.gemm(A, B))
    assert err <= (2e-5 if dtype == pgk.SPLIT_BF16 else 2e-2), err
