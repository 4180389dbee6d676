"""Host logic of the learned case selection (no GPU): feature rows, the
held-out shape generator and the regret summary."""
import math

import numpy as np

from paper_1801_04348_gb300 import costmodel, pgk


def test_feature_row_encodes_form_and_logs():
    p = pgk.params(16, 8, 4, 1, 0)
    f = costmodel.feature_row(1024, 64, 2048, p, pgk.F32)
    assert f == [10.0, 6.0, 11.0, 4.0, 3.0, 2.0, 0.0]
    q = pgk.params(16, 16, 8, 8, 8)
    assert costmodel.feature_row(64, 64, 64, q, pgk.F32)[-1] == 1.0
    t = pgk.params(128, 256, 4, 0, 0)
    assert costmodel.feature_row(64, 64, 64, t, pgk.BF16)[3:] == [7.0, 8.0, 2.0, 2.0]


def test_unseen_shapes_are_deduplicated_and_in_range():
    train = costmodel.training_shapes()
    assert len(train) == 517
    ev = costmodel.unseen_shapes(300, exclude=train)
    assert len(ev) == 300 and len(set(ev)) == 300
    assert not set(ev) & set(train)
    arr = np.asarray(ev)
    assert arr.min() >= 64 and arr.max() <= 16384 and np.all(arr % 16 == 0)


def test_summary_regret_and_time_saved():
    recs = [{"best_ms": 1.0, "model_ms": 1.0, "random_ms": 2.0, "default_ms": 1.5,
             "exhaustive_cost_ms": 10.0, "topk_cost_ms": 2.0},
            {"best_ms": 2.0, "model_ms": 2.2, "random_ms": 2.0, "default_ms": float("nan"),
             "exhaustive_cost_ms": 30.0, "topk_cost_ms": 3.0}]
    s = costmodel.summarize(recs, 3)
    assert math.isclose(s["model"]["geomean"], math.sqrt(1.0 * 1.1) - 1.0, rel_tol=1e-12)
    assert math.isclose(s["model"]["mean"], 0.05, rel_tol=1e-12)
    assert s["untuned_default"]["n"] == 1 and math.isclose(s["untuned_default"]["mean"], 0.5)
    assert math.isclose(s["tuning_time_saved"], 40.0 / 5.0)


def test_expected_random_min_equals_brute_force():
    """The exact expectation of the fastest of k random candidates equals the
    average over every k-subset (brute force), infeasible candidates excluded."""
    import itertools
    ms = [3.0, 1.0, float("inf"), 4.0, 1.5, 9.0, 2.5]
    feas = [x for x in ms if math.isfinite(x)]
    for k in range(1, len(feas) + 1):
        brute = np.mean([min(c) for c in itertools.combinations(feas, k)])
        assert math.isclose(costmodel.expected_random_min(ms, k), brute, rel_tol=1e-12)


def test_summary_by_k_uses_predictions_and_all_timings():
    recs = [{"best_ms": 1.0, "ms_all": [1.0, 2.0, 4.0], "pred_all": [3.0, 1.0, 2.0],
             "default_index": 2},
            {"best_ms": 2.0, "ms_all": [2.0, 3.0, float("inf")], "pred_all": [1.0, 2.0, float("inf")],
             "default_index": 1}]
    s1 = costmodel.summarize_k(recs, 1)
    # model top-1: candidate 1 (2.0 / 1.0) and candidate 0 (2.0 / 2.0)
    assert math.isclose(s1["model"]["mean"], 0.5, rel_tol=1e-12)
    # random single pick: mean of the feasible times over the best
    assert math.isclose(s1["random_k_expected"]["mean"], ((7.0 / 3.0) / 1.0 - 1 + 2.5 / 2.0 - 1) / 2)
    assert math.isclose(s1["untuned_default"]["mean"], (3.0 + 0.5) / 2)
    s2 = costmodel.summarize_k(recs, 2)
    assert math.isclose(s2["model"]["mean"], 0.5, rel_tol=1e-12)   # {1, 2} -> 2.0; {0, 1} -> 2.0
    assert math.isclose(s2["tuning_time_saved"], (7.0 + 5.0) / (6.0 + 5.0))
