"""Learned case selection on the GPU: the trained 7-64-64-1 network (weights
shipped with the package, trained by the library's own kernels on the timing
log of the tuning runs) against the method without it."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1801_04348_gb300 import costmodel, inputs, pgk

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(costmodel.__file__))


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def test_trained_network_beats_the_untrained_choices(dev):
    """Held-out shapes (log-uniform in [64, 16384], kept to <= 2048 here for
    time): the model's top-3 has small regret against exhaustive timing, less
    than the untuned default and than 3 random candidates."""
    cm = costmodel.CostModel.load(os.path.join(HERE, "costmodel_f32.json"))
    shapes = [s for s in costmodel.unseen_shapes(400, exclude=costmodel.training_shapes())
              if max(s) <= 2048][:24]
    recs, summ = costmodel.evaluate(cm, shapes, pgk.F32, dev, k=3, reps=2)
    print(summ)
    assert summ["model"]["geomean"] <= 0.05
    assert summ["model"]["geomean"] < summ["untuned_default"]["geomean"]
    assert summ["model"]["geomean"] < summ["random_k"]["geomean"]
    assert summ["tuning_time_saved"] > 3


@pytest.mark.parametrize("dtype,name", [(pgk.BF16, "bf16"), (pgk.SPLIT_BF16, "split")])
def test_trained_network_ranks_tensor_core_programs(dev, dtype, name):
    """The tensor-core forms have few tile programs, so the test takes the
    model's single best prediction (k = 1) on held-out shapes (<= 2048 here for
    time): its regret against exhaustive timing is small and below both the
    expected regret of one random program and the untuned default's."""
    cm = costmodel.CostModel.load(os.path.join(HERE, f"costmodel_{name}.json"))
    shapes = [s for s in costmodel.unseen_shapes(400, exclude=costmodel.training_shapes(dtype))
              if max(s) <= 2048][:24]
    recs, _ = costmodel.evaluate(cm, shapes, dtype, dev, k=1, reps=3)
    summ = costmodel.summarize_k(recs, 1)
    print(summ)
    assert summ["model"]["geomean"] <= 0.05
    assert summ["model"]["geomean"] < summ["random_k_expected"]["geomean"]
    assert summ["model"]["geomean"] < summ["untuned_default"]["geomean"]


def test_gemm_without_parameters_uses_the_learned_selection(dev):
    pgk.costmodel_load_file(pgk.F32, os.path.join(HERE, "costmodel_f32.json"), k=3)
    try:
        M, N, K = 1500, 1100, 700
        assert pgk.tune_cache_get(M, N, K, pgk.F32) is None
        A, B = inputs.gemm_operands(M, N, K, seed=4)
        C = torch.empty(M, N, device=dev)
        pgk.gemm(torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev), C, pgk.F32, None)
        torch.cuda.synchronize()
        chosen = pgk.tune_cache_get(M, N, K, pgk.F32)
        assert chosen is not None
        assert chosen.as_tuple() in [p.as_tuple() for p in costmodel.candidates(pgk.F32)]
        rows = np.linspace(0, M - 1, 16).astype(np.int64)
        err = oracle.rel_frobenius(C[torch.from_numpy(rows).to(dev)].cpu().numpy(),
                                   oracle.gemm(A, B, rows=rows))
        assert err <= 1e-5
    finally:
        pgk.costmodel_clear(pgk.F32)
