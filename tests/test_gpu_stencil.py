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


def test_transpose_order_2e14_sampled_rows(dev):
    """The timed workload (order 2^14, every point of the paper's grid): sampled rows
    of the transpose are the matching columns of the input, bit for bit."""
    n = 16384
    g = torch.Generator(device="cpu").manual_seed(14)
    a = torch.randint(-2 ** 31, 2 ** 31 - 1, (n, n), dtype=torch.int32, generator=g).to(dev)
    c = torch.empty(n, n, dtype=torch.int32, device=dev)
    rows = torch.from_numpy(np.r_[0, 1, np.linspace(2, n - 2, 30).astype(np.int64), n - 1]).to(dev)
    want = a[:, rows].t().cpu().numpy()
    for b0, b1 in TABLE_BLOCKS:
        for s in (2, 4, 8):
            c.fill_(-1)
            pgk.transpose(a, c, pgk.params(b0, b1, s))
            torch.cuda.synchronize()
            assert np.array_equal(c[rows].cpu().numpy(), want), (b0, b1, s)


def test_jacobi_2e27_windows(dev):
    """The timed workload (2^27 + 2 points, T = 4, every block and granularity of the
    grid at full size) against the oracle on windows: after T steps a point depends
    on the T points either side, so the oracle run on a window is exact everywhere
    but within T + 1 points of a cut that is not the array's own end."""
    n, steps = 2 ** 27 + 2, 4
    a = _jacobi_input(n, 27)
    starts = np.r_[0, np.linspace(5000, n - 5000, 14).astype(np.int64), n - 2048]
    refs = []
    for lo in starts:
        hi = min(lo + 2048, n)
        m = hi - lo
        sub = np.concatenate([a[lo:hi], a[n + lo:n + hi]])
        r = stencil.jacobi(sub, m, steps)
        v0 = 0 if lo == 0 else steps + 1
        v1 = m if hi == n else m - steps - 1
        refs.append((lo, v0, v1, r[v0:v1], r[m + v0:m + v1]))
    ad0 = torch.from_numpy(a).to(dev)
    for b in (16, 64, 128, 256):
        for s in (2, 8):
            ad = ad0.clone()
            pgk.jacobi(ad, n, steps, pgk.params(b, 1, s))
            torch.cuda.synchronize()
            for lo, v0, v1, r_first, r_second in refs:
                first = ad[lo + v0:lo + v1].cpu().numpy()
                second = ad[n + lo + v0:n + lo + v1].cpu().numpy()
                assert np.array_equal(first, r_first), (b, s, lo)
                assert np.array_equal(second, r_second), (b, s, lo)
