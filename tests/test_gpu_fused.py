"""The fused-conversion tensor-core programs (B1 = 64) for skinny products: A is
read in FP32 by the GEMM and converted to BF16 (hi and lo for the split form) in
shared memory, instead of in a separate pass.  The converted values are the
same, so every output equals the two-pass path on the library-prepared operands
bit for bit; the full skinny workload meets the forms' tolerances against the
FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_04348_gb300 import inputs, pgk

pytestmark = pytest.mark.gpu

# (form, fused program, two-pass program with the same products in the same order)
FORMS = [(pgk.SPLIT_BF16, (128, 64, 3), (128, 128, 3)),
         (pgk.BF16, (128, 64, 4), (128, 128, 6))]
TOL = {pgk.SPLIT_BF16: 2e-5, pgk.BF16: 2e-2}


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _two_pass(dev, form, prog, A, B, C0, beta):
    """The library's preparation entry points, then the prepared-operand GEMM."""
    M, K = A.shape
    N = B.shape[1]
    Kp = (K + 15) // 16 * 16
    a = torch.zeros(M, Kp, dtype=torch.int16, device=dev)
    b = torch.zeros(N, Kp, dtype=torch.int16, device=dev)
    C = C0.clone()
    if form == pgk.SPLIT_BF16:
        al, bl = torch.zeros_like(a), torch.zeros_like(b)
        pgk.split_bf16(A, a, al, 0)
        pgk.split_bf16(B, b, bl, 1)
        pgk.gemm_lowp(M, N, K, form, a, Kp, b, Kp, C, C.stride(0), A_lo=al, Bt_lo=bl, beta=beta,
                      prog=pgk.params(*prog, 0, 0))
    else:
        pgk.cvt_bf16(A, a, 0)
        pgk.cvt_bf16(B, b, 1)
        pgk.gemm_lowp(M, N, K, form, a, Kp, b, Kp, C, C.stride(0), beta=beta,
                      prog=pgk.params(*prog, 0, 0))
    return C


@pytest.mark.parametrize("form,fused,twopass", FORMS)
@pytest.mark.parametrize("M,N,K", [(300, 64, 1000), (129, 17, 200), (1, 1, 1), (256, 64, 64),
                                   (513, 40, 130), (1000, 64, 4099), (2000, 33, 3000)])
def test_fused_equals_two_pass(dev, form, fused, twopass, M, N, K):
    """One K slice (sr = 1); ragged M (tiles of 128 rows), N (one 64-wide tile), K
    (64-deep blocks, FP32 boxes of 32 columns past the end read as zeros), beta 0
    and 1.  A is a view with its row stride rounded up to 4 elements (16 bytes),
    as TMA needs."""
    A, B = inputs.gemm_operands(M, N, K, seed=M + 3 * N + 7 * K, dist="normal")
    lda = (K + 3) // 4 * 4
    Aw = torch.full((M, lda), float("nan"), device=dev)
    Aw[:, :K] = torch.from_numpy(A)
    At, Bt = Aw[:, :K], torch.from_numpy(B).to(dev)
    for beta in (0, 1):
        C0 = torch.randn(M, N, device=dev) if beta else torch.full((M, N), float("nan"), device=dev)
        ref = _two_pass(dev, form, twopass, At, Bt, C0, beta)
        C = C0.clone()
        pgk.gemm(At, Bt, C, form, pgk.params(*fused, 1, 0), beta=beta)
        torch.cuda.synchronize()
        pgk.check_device_error()
        assert not torch.isnan(C).any()
        assert torch.equal(C, ref), (form, M, N, K, beta)


@pytest.mark.parametrize("form,fused,twopass", FORMS)
def test_skinny_workload_16384x64x16384(dev, form, fused, twopass):
    """The skinny workload (M = K = 16384, N = 64, uniform[-1,1]): pgk_gemm without
    parameters takes the fused program (equal bit for bit to naming it), and 32
    sampled rows meet the form's tolerance against the FP64 oracle, row by row."""
    M, N, K = 16384, 64, 16384
    A, B = inputs.gemm_operands(M, N, K, seed=0)
    At, Bt = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    C = torch.empty(M, N, device=dev)
    Cn = torch.empty(M, N, device=dev)
    pgk.gemm(At, Bt, C, form, pgk.params(*fused, 0, 0))
    pgk.gemm(At, Bt, Cn, form, None)
    torch.cuda.synchronize()
    pgk.check_device_error()
    assert torch.equal(C, Cn)
    rows = np.linspace(0, M - 1, 32).astype(np.int64)
    ref = oracle.gemm(A, B, rows=rows)
    got = C[torch.from_numpy(rows).to(dev)].cpu().numpy().astype(np.float64)
    assert oracle.rel_frobenius(got, ref) <= TOL[form]
    per_row = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert per_row.max() <= TOL[form]


def test_fused_program_conditions(dev):
    """The case discussion refuses the fused program beyond N = 64 (INFEASIBLE);
    an A that TMA cannot read (row stride not a multiple of 16 bytes) is an
    ALIGNMENT error; the prepared-operand entry point has no FP32 A to read
    (UNSUPPORTED)."""
    prog = pgk.params(128, 64, 3, 0, 0)
    A = torch.randn(100, 130, device=dev)
    B = torch.randn(130, 65, device=dev)
    C = torch.empty(100, 65, device=dev)
    with pytest.raises(pgk.PgkError) as e:
        pgk.gemm(A, B, C, pgk.SPLIT_BF16, prog)
    assert e.value.status == 2
    Aw = torch.randn(100, 131, device=dev)
    with pytest.raises(pgk.PgkError) as e:
        pgk.gemm(Aw[:, :130], B[:, :64], C[:, :64], pgk.SPLIT_BF16, prog)
    assert e.value.status == 4
    a = torch.zeros(100, 144, dtype=torch.int16, device=dev)
    b = torch.zeros(64, 144, dtype=torch.int16, device=dev)
    with pytest.raises(pgk.PgkError) as e:
        pgk.gemm_lowp(100, 64, 130, pgk.SPLIT_BF16, a, 144, b, 144, C, 65, A_lo=a, Bt_lo=b, prog=prog)
    assert e.value.status == 3
    # without parameters an unaligned A takes a two-pass program instead
    Cd = torch.empty(100, 64, device=dev)
    pgk.gemm(Aw[:, :130], B[:, :64].contiguous(), Cd, pgk.SPLIT_BF16, None)
    torch.cuda.synchronize()
    ref = oracle.gemm(Aw[:, :130].contiguous().cpu().numpy(), B[:, :64].contiguous().cpu().numpy())
    assert oracle.rel_frobenius(Cd.cpu().numpy(), ref) <= 2e-5




@pytest.mark.parametrize("form,fused,twopass", FORMS)
@pytest.mark.parametrize("M,N,K,slices", [(300, 64, 1000, 2), (129, 17, 4099, 5), (1024, 64, 8192, 19),
                                          (200, 40, 130, 7)])
def test_k_slices(dev, form, fused, twopass, M, N, K, slices):
    """K split over slices (sr >= 2; the last slice shorter where the K blocks do
    not divide; more slices than K blocks give one block each): against the FP64
    oracle within the form's tolerance, against the one-slice program within the
    FP32 accumulation bound, and beta = 1 adds C once."""
    A, B = inputs.gemm_operands(M, N, K, seed=5 * M + N + K, dist="normal")
    lda = (K + 3) // 4 * 4
    Aw = torch.zeros((M, lda), device=dev)
    Aw[:, :K] = torch.from_numpy(A)
    At, Bt = Aw[:, :K], torch.from_numpy(B).to(dev)
    C1 = torch.empty(M, N, device=dev)
    pgk.gemm(At, Bt, C1, form, pgk.params(*fused, 1, 0))
    C0 = torch.randn(M, N, device=dev)
    Cs = C0.clone()
    pgk.gemm(At, Bt, Cs, form, pgk.params(*fused, slices, 0), beta=1)
    torch.cuda.synchronize()
    pgk.check_device_error()
    got = (Cs - C0).cpu().numpy().astype(np.float64)
    one = C1.cpu().numpy().astype(np.float64)
    ref = oracle.gemm(A, B)
    absab = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    assert oracle.rel_frobenius(got, ref) <= TOL[form]
    # one rounding per product term and per slice partial, plus the beta term
    bound = (3 * K + slices + 4) * 2.0 ** -24 * (absab + np.abs(one)) * 2.0 + 1e-6
    assert np.all(np.abs(got - one) <= bound + TOL[form] * np.abs(one))
    if form == pgk.SPLIT_BF16:
        assert np.all(np.abs(got - one) <= bound)


@pytest.mark.parametrize("form,fused,twopass", FORMS)
def test_few_row_tiles_take_k_slices(dev, form, fused, twopass):
    """4096 x 16 x 65536 (32 row tiles): without parameters the fused program
    splits K over slices to fill the SMs; the result meets the form's tolerance,
    row by row."""
    M, N, K = 4096, 16, 65536
    A, B = inputs.gemm_operands(M, N, K, seed=1)
    At, Bt = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    C = torch.empty(M, N, device=dev)
    pgk.gemm(At, Bt, C, form, None)
    torch.cuda.synchronize()
    pgk.check_device_error()
    rows = np.linspace(0, M - 1, 16).astype(np.int64)
    ref = oracle.gemm(A, B, rows=rows)
    got = C[torch.from_numpy(rows).to(dev)].cpu().numpy().astype(np.float64)
    per_row = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert per_row.max() <= TOL[form]


@pytest.mark.parametrize("form,fused,twopass", FORMS)
def test_every_tiny_shape(dev, form, fused, twopass):
    """Every M, N, K in [1, 9]: the fused program (one slice, two slices where K
    allows only one block so the count falls back to one, and the automatic count)
    equals the two-pass program bit for bit, beta 0."""
    import itertools
    for M, N, K in itertools.product(range(1, 10), repeat=3):
        A, B = inputs.gemm_operands(M, N, K, seed=M * 100 + N * 10 + K, dist="normal")
        Aw = torch.zeros((M, 12), device=dev)
        Aw[:, :K] = torch.from_numpy(A)
        At, Bt = Aw[:, :K], torch.from_numpy(B).to(dev)
        C0 = torch.full((M, N), float("nan"), device=dev)
        ref = _two_pass(dev, form, twopass, At, Bt, C0, 0)
        for slices in (1, 2, 0):
            C = C0.clone()
            pgk.gemm(At, Bt, C, form, pgk.params(*fused, slices, 0))
            assert torch.equal(C, ref), (form, M, N, K, slices)
    torch.cuda.synchronize()
    pgk.check_device_error()
