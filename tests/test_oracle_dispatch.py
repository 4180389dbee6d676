"""The GEMM family's case tree (Algorithms 1-2 with the counters of the kernel of
Fig. "cudamul") partitions the parameter space (Definition 2 (iii) and the
sibling-branch argument of the correctness lemma, Section 3.6)."""
import numpy as np

from oracle import comprehensive as co
from oracle import dispatch

# mock register counts per variant (the IR evaluation function of step S2)
def mock_regs(prog):
    fam, cap = prog["family"], prog["regopt"]
    if fam == "direct":
        return lambda e: 0 * e["B0"] + 16
    if fam == "paper":
        if prog["s"] == "s":
            return lambda e: np.minimum(20 + 6 * e["s"], 32) if cap else 20 + 6 * e["s"]
        return lambda e: 0 * e["B0"] + (26 if not cap else 26)
    return lambda e: 40 + e["sr"] * e["s"] + 0 * e["B0"]


BOX = co.make_box({
    "T": [256, 1024], "R": [24, 63, 255], "RB": [8192, 32768, 65536],
    "ZB": [0, 2048, 4096, 8192, 16384, 49152, 232448],
    "B0": [8, 16, 32], "B1": [8, 16, 32], "s": [1, 2, 4], "sr": [1], "BK": [8, 16, 32]})


def test_paper_family_leaves_partition_and_cover():
    leaves = dispatch.case_tree("paper", mock_regs, BOX)
    labels = {(dispatch.leaf_code(p), "1" in lam) for p, lam, _ in leaves}
    assert {(0, False), (1, False), (2, False)} <= labels      # 4a3a, 3b4a, 3b4b
    hits = dispatch.brute_force(leaves, BOX)
    assert max(len(h) for h in hits) <= 1                      # partition
    covered = np.array([len(h) == 1 for h in hits])
    e = BOX
    pre = e["B0"] <= e["B1"] * e["s"]
    thr = e["B0"] * e["B1"] <= e["T"]
    # a point is left uncovered only when no program in the family can run there
    assert not np.any(covered & ~(pre & thr))


def test_config1_grid_precondition_count():
    pts = [(b0, b1, s) for b0 in (8, 16, 32) for b1 in (8, 16, 32) for s in (1, 2, 4) if b0 <= b1 * s]
    assert len(pts) == 23
    excluded = {(b0, b1, s) for b0 in (8, 16, 32) for b1 in (8, 16, 32) for s in (1, 2, 4)} - set(pts)
    assert excluded == {(16, 8, 1), (32, 8, 1), (32, 8, 2), (32, 16, 1)}


def test_leaf_systems_match_paper_shape_on_smem():
    # with registers never binding, the three leaves are the paper's universal
    # shape: smem(s) <= Z_B ; smem(1) <= Z_B < smem(s) ; Z_B < smem(1)
    box = co.make_box({"T": [1024], "R": [255], "RB": [65536], "ZB": range(0, 40000, 512),
                       "B0": [8, 16], "B1": [16, 32], "s": [2, 4], "sr": [1], "BK": [8, 32]})
    leaves = dispatch.case_tree("paper", mock_regs, box)
    e = box
    sm_s = 4 * (e["B0"] * e["BK"] + e["BK"] * e["B1"] * e["s"])
    sm_1 = 4 * (e["B0"] * e["BK"] + e["BK"] * e["B1"])
    want = {0: sm_s <= e["ZB"], 1: (sm_1 <= e["ZB"]) & (e["ZB"] < sm_s), 2: e["ZB"] < sm_1}
    for code, region in want.items():
        got = np.zeros_like(region)
        for p, _, C in leaves:
            if dispatch.leaf_code(p) == code:
                got |= co.holds(C, box)
        assert np.array_equal(got, region), code


def test_rb_family_reduces_to_paper_form():
    box = co.make_box({"T": [1024], "R": [255], "RB": [65536], "ZB": [1024, 4096, 16384, 65536, 232448],
                       "B0": [8, 16], "B1": [8, 16], "s": [4, 8], "sr": [4, 8], "BK": [8, 16]})
    leaves = dispatch.case_tree("rb", mock_regs, box)
    hits = dispatch.brute_force(leaves, box)
    assert max(len(h) for h in hits) <= 1
    fams = {p["family"] for p, _, _ in leaves}
    assert fams == {"rb", "paper", "direct"}
