"""The offline case-table generator (Algorithms 1-2, product side): it regenerates
Fig. "compparkern"'s two cases, and its GEMM case table agrees at every box point
with the library's run-time walk (which the oracle checks independently)."""
import numpy as np

from paper_1801_04348_gb300 import build as pbuild
from paper_1801_04348_gb300 import casegen, pgk

REGS = [30, 34, 40, 56, 30, 32, 32, 40, 24, 24, 128]


def test_matrix_add_cases():
    spec = casegen.matrix_add_spec()
    box = casegen.make_box({"R": range(0, 40), "T": [64, 256, 1024], "B0": [1, 4, 16, 32],
                            "B1": [1, 8, 32]})
    leaves = casegen.generate(spec, box)
    assert sorted(n.prog["kernel"] for n, _ in leaves) == ["K1", "K2"]
    fits = box["B0"] * box["B1"] <= box["T"]
    k1 = casegen.leaf_region(leaves, lambda p: p["kernel"] == "K1")
    k2 = casegen.leaf_region(leaves, lambda p: p["kernel"] == "K2")
    assert np.array_equal(k1, fits & (box["R"] >= 14))
    assert np.array_equal(k2, fits & (box["R"] >= 10) & (box["R"] < 14))
    text = casegen.table_text(spec, leaves)
    assert "case 2" in text and "R < 14" in text


def test_gemm_table_matches_runtime_walk_and_lemma1():
    pbuild.build()
    spec = casegen.gemm_spec(REGS)
    box = casegen.make_box({"T": [256, 1024], "R": [40, 255], "RB": [8192, 65536],
                            "ZB": [0, 2048, 8192, 49152], "B0": [8, 16, 32], "B1": [8, 16, 32],
                            "s": [1, 2, 4], "BK": [8, 32]})
    leaves = casegen.generate(spec, box)
    n = len(box["T"])
    owner = np.full(n, -1)
    for k, (_, mask) in enumerate(leaves):
        assert not np.any(owner[mask] >= 0)          # leaves partition the box
        owner[mask] = k
    w, st = 3, 4
    for node, _ in leaves:                            # Lemma 1 (edge count per path)
        assert len(node.system) - 1 <= w + (w + 1) * st
    for i in range(n):
        pt = {k: int(v[i]) for k, v in box.items()}
        m = pgk.Machine(pt["T"], 49152, pt["ZB"], pt["RB"], 65536, pt["R"], 2048, 152, 32, 10, 3, 0)
        stt, c = pgk.select_case_regs(m, REGS, 64, 64, 64, pgk.F32,
                                      pgk.params(pt["B0"], pt["B1"], pt["s"], 1, pt["BK"]))
        if owner[i] < 0:
            assert stt == 2
            continue
        node = leaves[owner[i]][0]
        assert stt == 0
        want = 2 if not node.prog["cache"] else (0 if node.prog["s"] == "s" else 1)
        assert c.leaf == want and c.regopt == int(node.prog["cap"]), (pt, node.prog)
