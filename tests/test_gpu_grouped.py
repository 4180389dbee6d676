"""Grouped persistent GEMM: every problem matches the oracle and is bitwise equal
to the same tile variant launched alone (no split-K, identical per-tile order);
CUDA-graph replay reproduces the eager result."""
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


def make_group(dev, dims, seed0):
    host, dev_t = [], []
    for i, (M, N, K) in enumerate(dims):
        A, B = inputs.gemm_operands(int(M), int(N), int(K), seed=seed0 + 2 * i, dist="normal")
        host.append((A, B))
        dev_t.append((torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev),
                      torch.full((int(M), int(N)), float("nan"), device=dev)))
    return host, dev_t


def test_ragged_group_against_oracle_and_single_launches(dev):
    rng = np.random.default_rng(3)
    dims = rng.integers(1, 300, size=(40, 3))
    host, dt = make_group(dev, dims, 100)
    probs = pgk.make_problems(dt)
    for prog in pgk.grouped_variants():
        pgk.gemm_grouped(probs, pgk.F32, prog)
        torch.cuda.synchronize()
        for (A, B), (Ad, Bd, Cd) in zip(host, dt):
            C = Cd.cpu().numpy()
            assert_fp32_gemm(C, A, B)
            single = torch.empty_like(Cd)
            pgk.gemm(Ad, Bd, single, pgk.F32, prog)
            torch.cuda.synchronize()
            assert torch.equal(single, Cd), prog.as_tuple()


def test_config3_512_problems_graph_and_beta(dev):
    """512 GEMMs, M, N, K log-uniform in [32, 2048] rounded to multiples of 16
    (seed 0), normal(0,1) operands; sampled rows of every problem vs the oracle;
    graph replay equals eager; beta = 1 accumulates."""
    dims = inputs.log_uniform_dims(512, 0, 32, 2048, 16)
    host, dt = make_group(dev, dims, 1)
    probs = pgk.make_problems(dt)
    best, timings = pgk.autotune_grouped(probs, reps=2)
    assert all(np.isfinite(ms) for _, ms in timings)
    pgk.gemm_grouped(probs, pgk.F32, None)          # tuned default
    torch.cuda.synchronize()
    eager = [Cd.clone() for _, _, Cd in dt]
    for (A, B), (_, _, Cd) in zip(host, dt):
        rows = np.unique(np.linspace(0, A.shape[0] - 1, 6).astype(np.int64))
        assert_fp32_gemm(Cd.cpu().numpy()[rows], A, B, rows=rows)
    for _ in range(2):
        for _, _, Cd in dt:
            Cd.fill_(float("nan"))
        pgk.gemm_grouped(probs, pgk.F32, best, use_graph=1)
        torch.cuda.synchronize()
        for e, (_, _, Cd) in zip(eager, dt):
            assert torch.equal(e, Cd)
    pgk.gemm_grouped(probs, pgk.F32, best, beta=1)
    torch.cuda.synchronize()
    for e, (_, _, Cd) in zip(eager[:16], dt[:16]):
        assert torch.allclose(Cd, 2 * e, rtol=1e-6, atol=1e-4)


def test_invalid_problem_rejected(dev):
    A = torch.zeros(4, 4, device=dev)
    probs = pgk.make_problems([(A, A, A)])
    probs[0].lda = 1
    with pytest.raises(pgk.PgkError) as e:
        pgk.gemm_grouped(probs)
    assert e.value.status == 1


TC_FORMS = [(pgk.BF16, pgk.params(128, 128, 6, 0, 64)),
            (pgk.SPLIT_BF16, pgk.params(128, 128, 3, 0, 64)),
            (pgk.SPLIT_BF16, pgk.params(128, 128, 6, 0, 64)),
            (pgk.FP8_E4M3, pgk.params(128, 128, 6, 0, 128))]


@pytest.mark.parametrize("dtype,prog", TC_FORMS)
def test_tensor_core_group_equals_single_launches(dev, dtype, prog):
    """The tensor-core forms of a ragged group (sizes 1..300, odd K, unaligned
    strides): every problem equals pgk_gemm on it with the same tile program, bit
    for bit, for beta = 0 and 1 (packed operands at 128-row offsets, K zero-padded
    to the K block: the same tile arithmetic, and for FP8 the same 128 x 128 scale
    blocks, as a single launch)."""
    rng = np.random.default_rng(11)
    dims = rng.integers(1, 300, size=(30, 3))
    dims[0] = (1, 1, 1)
    dims[1] = (129, 257, 65)
    host, dt = make_group(dev, dims, 500)
    # one problem with padded strides (lda > K, ldb > N, ldc > N)
    M, N, K = 70, 90, 110
    A, B = inputs.gemm_operands(M, N, K, seed=77, dist="normal")
    Aw = torch.zeros(M, K + 5, device=dev)
    Aw[:, :K] = torch.from_numpy(A)
    Bw = torch.zeros(K, N + 3, device=dev)
    Bw[:, :N] = torch.from_numpy(B)
    Cw = torch.full((M, N + 7), float("nan"), device=dev)
    host.append((A, B))
    dt.append((Aw[:, :K], Bw[:, :N], Cw[:, :N]))
    probs = pgk.make_problems(dt)
    for beta in (0, 1):
        if beta:
            for _, _, Cd in dt:
                Cd.copy_(torch.randn_like(Cd))
        before = [Cd.clone() for _, _, Cd in dt]
        pgk.gemm_grouped(probs, dtype, prog, beta=beta)
        torch.cuda.synchronize()
        for (Ad, Bd, Cd), C0 in zip(dt, before):
            single = C0.clone()
            pgk.gemm(Ad, Bd, single, dtype, prog, beta=beta)
            torch.cuda.synchronize()
            assert torch.equal(single, Cd), (dtype, prog.as_tuple(), beta, tuple(Ad.shape), Bd.shape[1])
    assert torch.isnan(Cw[:, N:]).all()


def test_config3_512_problems_split_form(dev):
    """The 512-problem set in the split form: sampled rows of every problem within
    the split tolerance of the FP64 oracle."""
    dims = inputs.log_uniform_dims(512, 0, 32, 2048, 16)
    host, dt = make_group(dev, dims, 1)
    probs = pgk.make_problems(dt)
    pgk.gemm_grouped(probs, pgk.SPLIT_BF16, None)
    torch.cuda.synchronize()
    worst = 0.0
    for (A, B), (_, _, Cd) in zip(host, dt):
        rows = np.unique(np.linspace(0, A.shape[0] - 1, 4).astype(np.int64))
        ref = oracle.gemm(A, B, rows=rows)
        worst = max(worst, oracle.rel_frobenius(Cd.cpu().numpy()[rows].astype(np.float64), ref))
    assert worst <= 2e-5, worst
