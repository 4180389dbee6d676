"""Transposition and 1D Jacobi (Section 5) on the GPU: every case variant bit-exact
against the oracle, including ragged sizes and every leaf."""
import numpy as np
import pytest
import torch

from oracle import stencil
from paper_1801_04348_gb300 import pgk

pytestmark = pytest.mark.gpu

TABLE_BLOCKS = [(4, 32), (8, 32), (16, 32), (32, 32)]


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _words(rows, cols, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(-2 ** 31, 2 ** 31, size=(rows, cols), dtype=np.int64).astype(np.int32)


@pytest.mark.parametrize("rows,cols", [(512, 384), (1000, 777), (1, 1), (33, 2049), (300, 5)])
def test_transpose_every_block_and_granularity(dev, rows, cols):
    a = _words(rows, cols, rows + cols)
    ref = stencil.transpose(a)
    ad = torch.from_numpy(a).to(dev)
    for b0, b1 in TABLE_BLOCKS + [(8, 8), (1, 64)]:
        for s in (1, 2, 4, 8):
            c = torch.zeros(cols, rows, dtype=torch.int32, device=dev)
            pgk.transpose(ad, c, pgk.params(b0, b1, s))
            torch.cuda.synchronize()
            assert np.array_equal(c.cpu().numpy(), ref), (b0, b1, s)


def test_transpose_every_leaf_and_padded_strides(dev):
    rows, cols = 257, 300
    a = _words(rows, cols, 3)
    ref = stencil.transpose(a)
    src = torch.zeros(rows, cols + 7, dtype=torch.int32, device=dev)
    src[:, :cols] = torch.from_numpy(a).to(dev)
    m = pgk.machine_query(0)
    seen = set()
    for b0, b1, s in ((8, 32, 4), (16, 32, 2)):
        for zb in (m.smem_per_block_optin, 4 * b0 * (b1 * s + 1) - 4, 4 * b0 * (b1 + 1) - 4):
            mm = pgk.Machine(*[getattr(m, f) for f, _ in pgk.Machine._fields_])
            mm.smem_per_block_optin = zb
            st, c = pgk.select_case_transpose(mm, rows, cols, pgk.params(b0, b1, s))
            assert st == 0
            seen.add(c.leaf)
            dst = torch.full((cols, rows + 3), -1, dtype=torch.int32, device=dev)
            pgk.lib().pgk_transpose_case(pgk.ctypes.byref(c), rows, cols, src.data_ptr(), cols + 7,
                                         dst.data_ptr(), rows + 3, torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            out = dst.cpu().numpy()
            assert np.array_equal(out[:, :rows], ref)
            assert np.all(out[:, rows:] == -1)
    assert seen == {0, 1, 2}


def _jacobi_input(n, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(-2 ** 20, 2 ** 20, size=2 * n).astype(np.int32)


@pytest.mark.parametrize("n,steps", [(2 ** 15 + 2, 4), (3, 3), (1000, 7), (65537, 2)])
def test_jacobi_table_grid(dev, n, steps):
    """The paper's grid: blocks 16-256, granularity 2, 4, 8 (and 1)."""
    a = _jacobi_input(n, n)
    ref = stencil.jacobi(a, n, steps)
    for b in (16, 32, 64, 128, 256):
        for s in (1, 2, 4, 8):
            ad = torch.from_numpy(a).to(dev)
            pgk.jacobi(ad, n, steps, pgk.params(b, 1, s))
            torch.cuda.synchronize()
            assert np.array_equal(ad.cpu().numpy(), ref), (b, s)


def test_jacobi_every_leaf(dev):
    n, steps = 5000, 5
    a = _jacobi_input(n, 9)
    ref = stencil.jacobi(a, n, steps)
    m = pgk.machine_query(0)
    seen = set()
    for b, s in ((128, 2), (64, 8)):
        for zb in (m.smem_per_block_optin, 4 * (2 * s * b + 2) - 4, 4 * (2 * b + 2) - 4):
            mm = pgk.Machine(*[getattr(m, f) for f, _ in pgk.Machine._fields_])
            mm.smem_per_block_optin = zb
            st, c = pgk.select_case_jacobi(mm, n, pgk.params(b, 1, s))
            assert st == 0
            seen.add(c.leaf)
            ad = torch.from_numpy(a).to(dev)
            pgk.jacobi_case(c, ad, n, steps)
            torch.cuda.synchronize()
            assert np.array_equal(ad.cpu().numpy(), ref)
    assert seen == {0, 1, 2}
