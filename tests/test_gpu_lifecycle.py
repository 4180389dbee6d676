"""Library state across pgk_shutdown: the workspaces, the error word, cached
graphs and the allocation-free gradient's cached scratch address are released
and rebuilt on the next call, and every result is unchanged."""
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


def _run_all(dev):
    """One call of each workspace-using path; returns their outputs."""
    out = []
    A, B = inputs.gemm_operands(300, 200, 500, seed=41, dist="normal")
    At, Bt = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    for dtype, prog in ((pgk.SPLIT_BF16, pgk.params(256, 256, 3, 0, 0)),
                        (pgk.FP8_E4M3, pgk.params(128, 256, 4, 0, 0)),
                        (pgk.F32, pgk.params(16, 8, 8, 8, 16))):
        C = torch.full((300, 200), float("nan"), device=dev)
        pgk.gemm(At, Bt, C, dtype, prog)
        out.append(C)
    # skinny product with K slices (a slice workspace and the reduction)
    Bs = Bt[:, :40].contiguous()
    Cs = torch.full((300, 40), float("nan"), device=dev)
    pgk.gemm(At, Bs, Cs, pgk.SPLIT_BF16, pgk.params(128, 64, 3, 3, 0))
    out.append(Cs)
    # grouped: FP32 through a cached CUDA graph, and the split form
    trip = [(At, Bt, torch.zeros(300, 200, device=dev)), (At[:100], Bs, torch.zeros(100, 40, device=dev))]
    probs = pgk.make_problems(trip)
    pgk.gemm_grouped(probs, pgk.F32, pgk.params(16, 8, 8, 8, 8), use_graph=1)
    out += [trip[0][2].clone(), trip[1][2].clone()]
    pgk.gemm_grouped(probs, pgk.SPLIT_BF16, None)
    out += [trip[0][2].clone(), trip[1][2].clone()]
    # the cost-model gradient, allocating and allocation-free
    rng = np.random.default_rng(3)
    X = torch.from_numpy(rng.standard_normal((700, 7)).astype(np.float32)).to(dev)
    t = torch.from_numpy(rng.standard_normal(700).astype(np.float32)).to(dev)
    th = torch.from_numpy(inputs.he_uniform_mlp(2)).to(dev)
    for fn in (pgk.mlp_loss_grad, pgk.mlp_loss_grad_noalloc):
        g = torch.zeros(pgk.MLP_PARAMS, device=dev)
        loss = torch.zeros(1, device=dev)
        fn(X, t, th, g, loss)
        out += [g, loss]
    torch.cuda.synchronize()
    pgk.check_device_error()
    return [o.cpu() for o in out]


def test_results_survive_shutdown(dev):
    first = _run_all(dev)
    assert all(not torch.isnan(x).any() for x in first)
    pgk.shutdown()
    pgk.shutdown()                       # safe to call repeatedly
    second = _run_all(dev)
    for a, b in zip(first, second):
        assert torch.equal(a, b)
    assert torch.equal(second[-4], second[-2])   # allocating and allocation-free gradients
