"""Failure detection without a GPU fault: a bounded device wait that runs out is
reported as PGK_ERR_TIMEOUT through the error word and the context stays usable;
bad arguments are errors; the GEMM is capturable in a CUDA graph."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1801_04348_gb300 import inputs, pgk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def test_bounded_wait_reports_timeout_and_context_survives(dev):
    pgk.check_device_error()                       # clean start
    t0 = time.perf_counter()
    pgk.selftest_bounded_wait(50_000_000)          # 50 ms on a barrier nothing completes
    with pytest.raises(pgk.PgkError) as e:
        pgk.check_device_error()
    assert e.value.status == 6                     # PGK_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10
    pgk.check_device_error()                       # the word was cleared
    A, B = inputs.gemm_operands(64, 48, 80, seed=1)
    C = torch.zeros(64, 48, device=dev)
    pgk.gemm(torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev), C, pgk.SPLIT_BF16)
    torch.cuda.synchronize()
    pgk.check_device_error()
    assert oracle.rel_frobenius(C.cpu().numpy(), oracle.gemm(A, B)) < 2e-5


def test_argument_errors(dev):
    x = torch.zeros(8, 8, device=dev)
    with pytest.raises(pgk.PgkError) as e:
        pgk.gemm(x, x, x, pgk.F32, pgk.params(32, 8, 1))     # B0 > B1*s: no case
    assert e.value.status == 2
    with pytest.raises(pgk.PgkError) as e:
        pgk.gemm(x, x, x, pgk.BF16, pgk.params(128, 192, 4, 0, 0))   # no such tile
    assert e.value.status == 3
    odd = torch.zeros(8, 9, dtype=torch.int16, device=dev)
    c = torch.zeros(8, 8, device=dev)
    with pytest.raises(pgk.PgkError) as e:                   # row stride not a multiple of 16 B
        pgk.gemm_lowp(8, 8, 9, pgk.BF16, odd, 9, odd, 9, c, 8)
    assert e.value.status == 4


@pytest.mark.parametrize("form", [pgk.F32, pgk.SPLIT_BF16])
def test_gemm_in_cuda_graph(dev, form):
    M, N, K = 300, 260, 520
    A, B = inputs.gemm_operands(M, N, K, seed=2, dist="normal")
    Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    C = torch.zeros(M, N, device=dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pgk.gemm(Ad, Bd, C, form, stream=s)      # first call outside capture (workspaces)
        torch.cuda.synchronize()
        eager = C.clone()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            pgk.gemm(Ad, Bd, C, form, stream=s)
    C.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(C, eager)
