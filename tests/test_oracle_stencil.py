"""Pins for the transposition and 1D Jacobi oracles (Section 5), and the
library's case walk for both kernels against Algorithms 1-2 point by point."""
import numpy as np
import pytest

from oracle import comprehensive as co
from oracle import dispatch, stencil
from paper_1801_04348_gb300 import build as pbuild
from paper_1801_04348_gb300 import pgk


def test_transpose_definition():
    a = np.arange(12, dtype=np.int32).reshape(3, 4)
    c = stencil.transpose(a)
    assert c.shape == (4, 3)
    for i in range(3):
        for j in range(4):
            assert c[j, i] == a[i, j]
    assert np.array_equal(stencil.transpose(c), a)


def test_c_division_truncates_toward_zero():
    assert list(stencil.c_div3(np.array([7, -7, 8, -8, 0, 2, -2]))) == [2, -2, 2, -2, 0, 0, 0]


def test_jacobi_hand_example():
    # n = 5: interior p = 0, 1, 2.  Step 0 writes the second half from the first.
    a = np.array([3, 6, 9, 12, 0, 0, 0, 0, 0, 0], dtype=np.int32)
    r = stencil.jacobi(a, 5, 1)
    assert list(r) == [3, 6, 9, 12, 0, 0, 6, 9, 7, 0]   # (3+6+9)/3, (6+9+12)/3, (9+12+0)/3
    r2 = stencil.jacobi(a, 5, 2)                        # step 1 writes the first half back
    assert list(r2[:5]) == [3, (0 + 6 + 9) // 3, (6 + 9 + 7) // 3, (9 + 7 + 0) // 3, 0]


def test_jacobi_invariants():
    n = 40
    const = np.full(2 * n, -9, dtype=np.int32)
    assert np.array_equal(stencil.jacobi(const, n, 7), const)
    ramp = np.concatenate([np.arange(n) * 3, np.arange(n) * 3]).astype(np.int32)
    # the average of three consecutive terms of an arithmetic sequence is the middle one
    assert np.array_equal(stencil.jacobi(ramp, n, 5), ramp)


REGS = [20, 22, 26, 34, 14]   # cached s = 1, 2, 4, 8; direct


def _regs_of(prog):
    if not prog["cache"]:
        return lambda e: 0 * e["B0"] + REGS[4]
    if prog["s"] == "s":
        def f(e):
            out = np.zeros_like(e["s"])
            for sv, si in ((1, 0), (2, 1), (4, 2), (8, 3)):
                out = np.where(e["s"] == sv, REGS[si], out)
            return out
        return f
    return lambda e: 0 * e["B0"] + REGS[0]


@pytest.mark.parametrize("kind", ["transpose", "jacobi"])
def test_library_walk_matches_oracle_tree(kind):
    pbuild.build()
    box = co.make_box({"T": [256, 1024], "R": [24, 255], "RB": [4096, 65536],
                       "ZB": [0, 128, 1024, 4096, 16384, 232448],
                       "B0": [4, 8, 32, 128], "B1": [1, 8, 32] if kind == "transpose" else [1],
                       "s": [1, 2, 4, 8]})
    leaves = dispatch.stencil_case_tree(kind, _regs_of, box)
    hits = dispatch.brute_force(leaves, box)
    n = len(next(iter(box.values())))
    seen = set()
    for i in range(n):
        pt = {k: int(v[i]) for k, v in box.items()}
        m = pgk.Machine(pt["T"], 49152, pt["ZB"], pt["RB"], 65536, pt["R"], 2048, 152, 32, 10, 3, 0)
        prog = pgk.params(pt["B0"], pt["B1"], pt["s"])
        if kind == "transpose":
            st, c = pgk.select_case_transpose(m, 64, 64, prog, regs=REGS)
        else:
            st, c = pgk.select_case_jacobi(m, 1000, prog, regs=REGS)
        assert len(hits[i]) <= 1
        if not hits[i]:
            assert st == 2, (pt, st)
            continue
        assert st == 0, (pt, st, pgk.last_error())
        p, lam, _ = leaves[hits[i][0]]
        want = 2 if not p["cache"] else (0 if p["s"] == "s" else 1)
        assert c.leaf == want, (pt, c.leaf, p)
        seen.add(c.leaf)
    assert seen == {0, 1, 2}


def test_jacobi_leaf_systems_are_the_papers():
    # with registers never binding the leaves are Fig. "1dj"'s three systems
    # (in bytes: 4 (2 s B + 2) <= Z_B ; 4 (2 B + 2) <= Z_B < 4 (2 s B + 2) ; Z_B < 4 (2 B + 2))
    box = co.make_box({"T": [1024], "R": [255], "RB": [65536], "ZB": range(0, 20000, 64),
                       "B0": [16, 64, 128, 256], "B1": [1], "s": [2, 4, 8]})
    leaves = dispatch.stencil_case_tree("jacobi", _regs_of, box)
    e = box
    want = {0: 4 * (2 * e["s"] * e["B0"] + 2) <= e["ZB"],
            1: (4 * (2 * e["B0"] + 2) <= e["ZB"]) & (e["ZB"] < 4 * (2 * e["s"] * e["B0"] + 2)),
            2: e["ZB"] < 4 * (2 * e["B0"] + 2)}
    for code, region in want.items():
        got = np.zeros_like(region)
        for p, _, C in leaves:
            pc = 2 if not p["cache"] else (0 if p["s"] == "s" else 1)
            if pc == code:
                got |= co.holds(C, box)
        assert np.array_equal(got, region), code
