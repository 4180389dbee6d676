"""Pins for the Algorithms 1-2 oracle: it must reproduce the case systems the
paper prints for its own examples (Fig. "compparkern", Section 1; Fig. "1dj" and
Fig. "transpose", Section 5) and satisfy Definition 2 (coverage, partition)."""
import json
import os
import re

import numpy as np

from oracle import comprehensive as co

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "printed_case_systems.json")))


def _printed(example, program, box):
    """Union over the printed systems of `program`, evaluated on the box.  Each
    inequality is a chain a op b [op c] with op in {<=, <}; terms are products
    and sums of symbols and integers."""
    def term(t):
        val = 0
        for summand in t.split("+"):
            prod = 1
            for f in summand.split("*"):
                f = f.strip()
                prod = prod * (int(f) if f.isdigit() else box[f])
            val = val + prod
        return val

    out = np.zeros(len(next(iter(box.values()))), dtype=bool)
    for system in GOLDEN[example]["cases"][program]:
        ok = np.ones_like(out)
        for ineq in system:
            parts = re.split(r"(<=|<)", ineq)
            for i in range(0, len(parts) - 2, 2):
                a, op, b = term(parts[i]), parts[i + 1], term(parts[i + 2])
                ok &= (a <= b) if op == "<=" else (a < b)
        out |= ok
    return out


def _region(leaves, prog_pred, box):
    ok = np.zeros(len(next(iter(box.values()))), dtype=bool)
    for prog, _, C in leaves:
        if prog_pred(prog):
            ok |= co.holds(C, box)
    return ok


def _matrix_add_tree():
    # Two machine parameters R (registers per thread) and T (threads per block),
    # program parameters B0, B1; registers 14 for K1, 10 after reducing granularity.
    counters = {
        "threads": co.Counter("threads", "resource", "T", lambda p: ("B0 B1", lambda e: e["B0"] * e["B1"]), ()),
        "regs": co.Counter("regs", "resource", "R",
                           lambda p: (str(p["regs"]), lambda e, r=p["regs"]: 0 * e["R"] + r), ("3b",)),
    }
    strategies = {"3b": co.Strategy("3b", False, lambda p: {"kernel": "K2", "regs": 10})}
    box = co.make_box({"R": range(0, 40), "T": [64, 256, 512, 1024], "B0": [1, 2, 4, 8, 16, 32], "B1": [1, 2, 4, 8, 16, 32]})
    Q = co.initial_quintuple({"kernel": "K1", "regs": 14}, ["3b"], ["threads", "regs"], [])
    return co.comprehensive_optimization(Q, counters, strategies, box), box


def test_matrix_add_example_reproduces_C1_C2():
    leaves, box = _matrix_add_tree()
    assert sorted(p["kernel"] for p, _, _ in leaves) == ["K1", "K2"]
    k1 = _region(leaves, lambda p: p["kernel"] == "K1", box)
    k2 = _region(leaves, lambda p: p["kernel"] == "K2", box)
    assert np.array_equal(k1, _printed("matrix_add", "K1", box))            # C1
    assert np.array_equal(k2, _printed("matrix_add", "K2", box))            # C2
    assert not np.any(k1 & k2)


def _three_case_tree(smem_s, smem_1, regs_full, regs_reduced, reg_sigma):
    counters = {
        "regs": co.Counter("regs", "resource", "RB",
                           lambda p: ("regs", lambda e, r=p["regs"]: 0 * e["RB"] + r), reg_sigma),
        "smem": co.Counter("smem", "resource", "ZB", lambda p: ("smem", p["smem"]), ("3b", "4b")),
    }

    def gran(p):
        return {"case": "3b4a" if p["case"] == "4a3a" else p["case"], "smem": smem_1, "regs": regs_reduced}

    def nocache(p):
        return {"case": "3b4b", "smem": lambda e: 0 * e["ZB"], "regs": p["regs"]}

    strategies = {"3b": co.Strategy("3b", False, gran), "4b": co.Strategy("4b", False, nocache)}
    box = co.make_box({"ZB": range(0, 300, 2), "RB": range(0, 14), "s": [2, 4, 8], "B": [4, 8, 16],
                       "B0": [2, 4, 8], "B1": [2, 4, 8]})
    Q = co.initial_quintuple({"case": "4a3a", "smem": smem_s, "regs": regs_full},
                             ["3b", "4b"], ["regs", "smem"], [])
    return co.comprehensive_optimization(Q, counters, strategies, box), box


def test_jacobi_example_three_cases():
    # Fig. "1dj": 2sB+2 <= Z_B ; 2B+2 <= Z_B < 2sB+2 ; Z_B < 2B+2 ; all with 9 <= R_B
    leaves, box = _three_case_tree(lambda e: 2 * e["s"] * e["B"] + 2, lambda e: 2 * e["B"] + 2, 9, 9, ())
    for case in ("4a3a", "3b4a", "3b4b"):
        got = _region(leaves, lambda p, c=case: p["case"] == c, box)
        assert np.array_equal(got, _printed("jacobi", case, box)), case


def test_transpose_example_printed_systems_are_sound():
    # Fig. "transpose": registers 6, or 5 once granularity is reduced; reducing
    # granularity also serves the register counter.  Every printed system must lie
    # inside the region the algorithm assigns to that program, and the three
    # regions must be disjoint.
    leaves, box = _three_case_tree(lambda e: 2 * e["s"] * e["B0"] * e["B1"],
                                   lambda e: 2 * e["B0"] * e["B1"], 6, 5, ("3b",))
    RB = box["RB"]
    r1 = _region(leaves, lambda p: p["case"] == "4a3a", box)
    r2 = _region(leaves, lambda p: p["case"] == "3b4a", box)
    r3 = _region(leaves, lambda p: p["case"] == "3b4b", box)
    assert np.array_equal(r1, _printed("transpose", "4a3a", box))
    assert not np.any(_printed("transpose", "3b4a", box) & ~r2)
    assert not np.any(_printed("transpose", "3b4b", box) & ~r3)
    assert not np.any(r1 & r2) and not np.any(r1 & r3) and not np.any(r2 & r3)
    # coverage (Definition 2 (iii)): every point with at least 5 registers has a case
    assert np.array_equal(r1 | r2 | r3, RB >= 5)


def test_tree_height_bound():
    # Lemma 1 bounds the height by the strategies w and counters s + t.  Counting
    # one edge per constraint, a path holds at most w refuse edges and at most
    # s + t accept edges before, between and after them: w + (w + 1)(s + t).
    leaves, _ = _matrix_add_tree()
    w, st = 1, 2
    for _, _, C in leaves:
        assert len(C) <= w + (w + 1) * st
    assert co.tree_height_bound(w, st, 0) == 2


def test_stack_push_convention():
    s = ["s1", "s2"]
    co.push_sequence(s, ["t1", "t2", "t3"])
    assert s == ["t3", "t2", "t1", "s1", "s2"]
