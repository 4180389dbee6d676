"""int32 GEMM modulo 2^32 (the paper's data type): every variant bit-exact
against the oracle, full-range operands (products and sums overflow)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_04348_gb300 import pgk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _ops(M, N, K, seed):
    rng = np.random.default_rng(seed)
    A = rng.integers(-2 ** 31, 2 ** 31, size=(M, K), dtype=np.int64).astype(np.int32)
    B = rng.integers(-2 ** 31, 2 ** 31, size=(K, N), dtype=np.int64).astype(np.int32)
    return A, B


def _run(dev, A, B, prog, beta=0, C0=None):
    C = torch.from_numpy(C0).to(dev) if C0 is not None else torch.zeros(
        A.shape[0], B.shape[1], dtype=torch.int32, device=dev)
    pgk.gemm_i32(torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev), C, prog, beta=beta)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def _progs():
    out = [pgk.params(b0, b1, s) for b0 in (8, 16, 32) for b1 in (8, 16, 32) for s in (1, 2, 4)
           if b0 <= b1 * s]
    out += [pgk.params(4, 16, 4), pgk.params(8, 64, 2), pgk.params(16, 16, 8)]
    for i in range(pgk.num_variants()):
        v = pgk.variant_info_get(i)
        if v.family == pgk.FAM_RB_I32:
            out.append(pgk.params(v.B0, v.B1, v.s, v.sr, v.tile))
    return out


@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (129, 77, 301), (1, 1, 1), (5, 300, 33)])
def test_every_variant_bit_exact(dev, M, N, K):
    A, B = _ops(M, N, K, M + N + K)
    ref = oracle.gemm_i32(A, B)
    for p in _progs():
        assert np.array_equal(_run(dev, A, B, p), ref), p.as_tuple()


def test_beta_and_every_leaf(dev):
    M, N, K = 97, 131, 67
    A, B = _ops(M, N, K, 7)
    C0 = np.random.default_rng(8).integers(-2 ** 31, 2 ** 31, size=(M, N), dtype=np.int64).astype(np.int32)
    ref = oracle.gemm_i32(A, B, C0=C0, beta=1)
    m = pgk.machine_query(0)
    seen = set()
    for b0, b1, s in ((8, 16, 2), (16, 16, 4), (32, 8, 4)):
        for zb in (m.smem_per_block_optin, 4 * (b0 * b0 + b0 * b1 * s) - 4, 4 * (b0 * b0 + b0 * b1) - 4):
            mm = pgk.Machine(*[getattr(m, f) for f, _ in pgk.Machine._fields_])
            mm.smem_per_block_optin = zb
            st, c = pgk.select_case(mm, M, N, K, pgk.I32, pgk.params(b0, b1, s), raise_on_error=False)
            assert st == 0
            assert c.family in (pgk.FAM_PAPER_I32, pgk.FAM_DIRECT_I32)
            seen.add(c.leaf)
            Ct = torch.from_numpy(C0.copy()).to(dev)
            pgk.gemm_case(c, torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev), Ct, beta=1)
            torch.cuda.synchronize()
            assert np.array_equal(Ct.cpu().numpy(), ref)
    assert seen == {0, 1, 2}


def test_split_k_int32(dev):
    A, B = _ops(48, 80, 9000, 21)
    ref = oracle.gemm_i32(A, B)
    for p in _progs():
        if p.sr > 1:
            assert np.array_equal(_run(dev, A, B, p), ref), p.as_tuple()
