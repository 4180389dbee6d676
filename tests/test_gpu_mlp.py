"""Cost-model kernels (forward, loss gradient, Adam) against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import mlp
from paper_1801_04348_gb300 import inputs, pgk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _data(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 7)).astype(np.float32), rng.standard_normal(n).astype(np.float32)


def _theta(seed=0):
    th = inputs.he_uniform_mlp(seed)
    th = th + np.random.default_rng(seed + 1).normal(0, 0.05, th.size).astype(np.float32)
    return th.astype(np.float32)


def test_forward_matches_oracle(dev):
    X, _ = _data(1000, 1)
    th = _theta()
    y = torch.zeros(1000, device=dev)
    pgk.mlp_forward(torch.from_numpy(X).to(dev), torch.from_numpy(th).to(dev), y)
    torch.cuda.synchronize()
    ref, _ = mlp.forward(th.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [1, 17, 256, 5000])
def test_gradient_matches_oracle(dev, n):
    X, t = _data(n, 2 + n)
    th = _theta(3)
    Xd, td, thd = (torch.from_numpy(a).to(dev) for a in (X, t, th))
    g = torch.zeros(pgk.MLP_PARAMS, device=dev)
    loss = torch.zeros(1, device=dev)
    pgk.mlp_loss_grad(Xd, td, thd, g, loss)
    torch.cuda.synchronize()
    L, gref = mlp.loss_and_grad(th.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert abs(loss.item() - L) <= 1e-5 * abs(L)
    gg = g.cpu().numpy().astype(np.float64)
    for name, shape in mlp.SHAPES:
        a = mlp.unpack(gg)[name]
        b = mlp.unpack(gref)[name]
        assert np.linalg.norm(a - b) <= 1e-4 * max(np.linalg.norm(b), 1e-12), name
    # deterministic: a second call is bitwise identical
    g2 = torch.zeros_like(g)
    pgk.mlp_loss_grad(Xd, td, thd, g2, loss)
    torch.cuda.synchronize()
    assert torch.equal(g, g2)


def test_minibatch_indices(dev):
    X, t = _data(300, 5)
    th = _theta(4)
    idx = np.random.default_rng(6).permutation(300)[:64].astype(np.int32)
    g = torch.zeros(pgk.MLP_PARAMS, device=dev)
    loss = torch.zeros(1, device=dev)
    pgk.mlp_loss_grad(torch.from_numpy(X).to(dev), torch.from_numpy(t).to(dev),
                      torch.from_numpy(th).to(dev), g, loss, idx=torch.from_numpy(idx).to(dev))
    torch.cuda.synchronize()
    L, gref = mlp.loss_and_grad(th.astype(np.float64), X[idx].astype(np.float64), t[idx].astype(np.float64))
    assert abs(loss.item() - L) <= 1e-5 * L
    assert np.linalg.norm(g.cpu().numpy() - gref) <= 1e-4 * np.linalg.norm(gref)


def test_adam_steps_match_oracle(dev):
    th = _theta(7).astype(np.float64)
    rng = np.random.default_rng(8)
    thd = torch.from_numpy(th.astype(np.float32)).to(dev)
    m = torch.zeros_like(thd)
    v = torch.zeros_like(thd)
    mo = np.zeros_like(th)
    vo = np.zeros_like(th)
    to = th.astype(np.float32).astype(np.float64)
    for step in range(1, 4):
        g = rng.normal(size=th.size).astype(np.float32)
        pgk.mlp_adam(thd, torch.from_numpy(g).to(dev), m, v, step)
        to, mo, vo = mlp.adam_step(to, g.astype(np.float64), mo, vo, step)
    torch.cuda.synchronize()
    assert np.max(np.abs(thd.cpu().numpy() - to)) <= 1e-6


def test_training_reduces_loss(dev):
    """A few hundred Adam steps on a smooth synthetic target cut the loss."""
    rng = np.random.default_rng(9)
    X = rng.uniform(-1, 1, (2048, 7)).astype(np.float32)
    t = (X @ rng.normal(size=7) + np.sin(3 * X[:, 0])).astype(np.float32)
    Xd, td = torch.from_numpy(X).to(dev), torch.from_numpy(t).to(dev)
    th = torch.from_numpy(inputs.he_uniform_mlp(0)).to(dev)
    m, v = torch.zeros_like(th), torch.zeros_like(th)
    g = torch.zeros_like(th)
    loss = torch.zeros(1, device=dev)
    pgk.mlp_loss_grad(Xd, td, th, g, loss)
    torch.cuda.synchronize()
    first = loss.item()
    step = 0
    for epoch in range(30):
        perm = torch.from_numpy(rng.permutation(2048).astype(np.int32)).to(dev)
        for b in range(0, 2048, 256):
            step += 1
            pgk.mlp_loss_grad(Xd, td, th, g, loss, idx=perm[b:b + 256])
            pgk.mlp_adam(th, g, m, v, step, lr=3e-3)
    pgk.mlp_loss_grad(Xd, td, th, g, loss)
    torch.cuda.synchronize()
    assert loss.item() < 0.05 * first
