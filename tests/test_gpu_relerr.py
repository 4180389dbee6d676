"""FP64 error-measurement reduction on the GPU against numpy's FP64 sums."""
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


@pytest.mark.parametrize("R,Cc", [(1, 1), (37, 1001), (2048, 2048)])
def test_relerr_sums(dev, R, Cc):
    ref = inputs.normal((R, Cc), 1).astype(np.float64) * 3.0
    C = (ref + inputs.normal((R, Cc), 2) * 1e-3).astype(np.float32)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    pgk.relerr(torch.from_numpy(C).to(dev), torch.from_numpy(ref).to(dev), out)
    torch.cuda.synchronize()
    num = np.sum((C.astype(np.float64) - ref) ** 2)
    den = np.sum(ref ** 2)
    got = out.cpu().numpy()
    assert abs(got[0] - num) <= 1e-12 * num + 1e-300
    assert abs(got[1] - den) <= 1e-12 * den


def test_relerr_row_index_and_determinism(dev):
    C = inputs.uniform((100, 64), 3)
    rows = np.array([5, 99, 0, 42], dtype=np.int64)
    ref = C[rows].astype(np.float64) * 1.5
    Cd = torch.from_numpy(C).to(dev)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    pgk.relerr(Cd, torch.from_numpy(ref).to(dev), out, row_index=torch.from_numpy(rows).to(dev))
    torch.cuda.synchronize()
    first = out.clone()
    num = np.sum((C[rows].astype(np.float64) - ref) ** 2)
    assert abs(out[0].item() - num) <= 1e-12 * num
    pgk.relerr(Cd, torch.from_numpy(ref).to(dev), out, row_index=torch.from_numpy(rows).to(dev))
    torch.cuda.synchronize()
    assert torch.equal(first, out)
