"""The allocation-free gradient entry point (pgk_mlp_loss_grad_noalloc) gives the
same result as pgk_mlp_loss_grad, on two calls in a row.

It exists for callers that cannot allocate device memory where they need the
gradient: real-time training loops that forbid allocation after start-up, and
host applications whose device memory belongs to their own pool allocator.  Its
scratch is a static device array of the library.  Both entry points launch the
same kernels with the same fixed reduction order, so the results must be equal
bit for bit.  This file is collected last so that a run stopping at the first
failure has already run every other test; it passes alone in a fresh process
too."""
import numpy as np
import pytest
import torch

from paper_1801_04348_gb300 import inputs, pgk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _case(n, seed, dev):
    rng = np.random.default_rng(seed)
    X = torch.from_numpy(rng.standard_normal((n, 7)).astype(np.float32)).to(dev)
    t = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
    th = torch.from_numpy(inputs.he_uniform_mlp(seed)).to(dev)
    return X, t, th


def test_noalloc_matches_allocating_entry_point_twice(dev):
    for n, seed in ((300, 1), (2048, 2)):          # two calls in a row, reusing the scratch
        X, t, th = _case(n, seed, dev)
        g_ref = torch.zeros(pgk.MLP_PARAMS, device=dev)
        l_ref = torch.zeros(1, device=dev)
        pgk.mlp_loss_grad(X, t, th, g_ref, l_ref)
        g = torch.full((pgk.MLP_PARAMS,), float("nan"), device=dev)
        loss = torch.full((1,), float("nan"), device=dev)
        pgk.mlp_loss_grad_noalloc(X, t, th, g, loss)
        torch.cuda.synchronize()
        assert torch.equal(g, g_ref)
        assert torch.equal(loss, l_ref)


def test_noalloc_minibatch_indices(dev):
    X, t, th = _case(1000, 3, dev)
    idx = torch.from_numpy(np.random.default_rng(4).permutation(1000)[:256].astype(np.int32)).to(dev)
    g_ref = torch.zeros(pgk.MLP_PARAMS, device=dev)
    l_ref = torch.zeros(1, device=dev)
    pgk.mlp_loss_grad(X, t, th, g_ref, l_ref, idx=idx)
    g = torch.zeros_like(g_ref)
    loss = torch.zeros_like(l_ref)
    pgk.mlp_loss_grad_noalloc(X, t, th, g, loss, idx=idx)
    torch.cuda.synchronize()
    assert torch.equal(g, g_ref)
    assert torch.equal(loss, l_ref)


def test_noalloc_rejects_batches_beyond_the_limit(dev):
    X, t, th = _case(2049, 5, dev)
    g = torch.zeros(pgk.MLP_PARAMS, device=dev)
    loss = torch.zeros(1, device=dev)
    with pytest.raises(pgk.PgkError) as e:
        pgk.mlp_loss_grad_noalloc(X, t, th, g, loss)
    assert e.value.status == 1 and "2048" in str(e.value)
