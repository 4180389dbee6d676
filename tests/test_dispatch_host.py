"""The library's case walk (pgk_select_case_regs, host code) agrees at every
point with the oracle's Algorithms 1-2 tree for the GEMM family, evaluated by
brute force (each leaf's conjunction checked separately), on mock machines."""
import numpy as np
import pytest

from oracle import comprehensive as co
from oracle import dispatch
from paper_1801_04348_gb300 import build as pbuild
from paper_1801_04348_gb300 import pgk

# register counts per class: paper s=1,2,4,8 ; capped ; direct ; direct capped ; rb
TABLES = {
    "small": [30, 34, 40, 56, 30, 32, 32, 40, 24, 24, 128],
    "heavy": [70, 80, 90, 120, 60, 62, 63, 64, 80, 40, 168],
}
S_INDEX = {1: 0, 2: 1, 4: 2, 8: 3}


def regs_fn(table):
    def regs_of(prog):
        fam, cap = prog["family"], prog["regopt"]
        if fam == "direct":
            return lambda e: 0 * e["B0"] + table[9 if cap else 8]
        if fam == "rb":
            return lambda e: 0 * e["B0"] + table[10]
        if prog["s"] == "s":
            def f(e):
                out = np.zeros_like(e["s"])
                for sv, si in S_INDEX.items():
                    out = np.where(e["s"] == sv, table[si + (4 if cap else 0)], out)
                return out
            return f
        return lambda e, s=prog["s"]: 0 * e["B0"] + table[S_INDEX[s] + (4 if cap else 0)]
    return regs_of


@pytest.fixture(scope="module")
def built():
    pbuild.build()
    return pgk.lib()


def _compare(box, family, table, rb_ok=lambda p: True):
    leaves = dispatch.case_tree(family, regs_fn(table), box)
    hits = dispatch.brute_force(leaves, box)
    n = len(next(iter(box.values())))
    checked = 0
    for i in range(n):
        pt = {k: int(v[i]) for k, v in box.items()}
        if not rb_ok(pt):
            continue
        m = pgk.Machine(pt["T"], 49152, pt["ZB"], pt["RB"], 65536, pt["R"], 2048, 152, 32, 10, 3, 0)
        prog = pgk.params(pt["B0"], pt["B1"], pt["s"], pt["sr"], pt["BK"])
        st, c = pgk.select_case_regs(m, table, 64, 64, 64, pgk.F32, prog)
        assert len(hits[i]) <= 1
        if not hits[i]:
            assert st == 2, (pt, st)                     # INFEASIBLE
            continue
        assert st == 0, (pt, st, pgk.last_error())
        p, lam, _ = leaves[hits[i][0]]
        assert c.leaf == dispatch.leaf_code(p), (pt, c.leaf, p)
        assert c.regopt == int("1" in lam), (pt, lam)
        want_fam = {"paper": pgk.FAM_PAPER, "rb": pgk.FAM_RB, "direct": pgk.FAM_DIRECT}[p["family"]]
        assert c.family == want_fam
        checked += 1
    return checked


@pytest.mark.parametrize("tname", list(TABLES))
def test_paper_family_walk_matches_oracle(built, tname):
    box = co.make_box({"T": [256, 1024], "R": [63, 255], "RB": [16384, 32768, 65536],
                       "ZB": [0, 1024, 4096, 16384, 49152, 232448],
                       "B0": [8, 16, 32], "B1": [8, 16, 32], "s": [1, 2, 4, 8], "sr": [1],
                       "BK": [8, 16, 32]})
    assert _compare(box, "paper", TABLES[tname]) > 100


def test_rb_family_walk_matches_oracle(built):
    compiled = set()
    for i in range(pgk.num_variants()):
        v = pgk.variant_info_get(i)
        if v.family == pgk.FAM_RB:
            compiled.add((v.B0, v.B1, v.sr, v.s, v.tile))
    box = co.make_box({"T": [256, 1024], "R": [255], "RB": [32768, 65536],
                       "ZB": [0, 4096, 16384, 65536, 232448],
                       "B0": [8, 16, 32], "B1": [8, 16, 32], "s": [4, 8], "sr": [4, 8], "BK": [8, 16]})
    ok = lambda p: (p["B0"], p["B1"], p["sr"], p["s"], p["BK"]) in compiled
    assert _compare(box, "rb", TABLES["small"], ok) > 20
    assert _compare(box, "rb", TABLES["heavy"], ok) > 5


def test_real_gb300_like_machine_picks_4a3a(built):
    m = pgk.Machine(1024, 49152, 232448, 65536, 65536, 255, 2048, 152, 32, 10, 3, 0)
    for b0 in (8, 16, 32):
        for b1 in (8, 16, 32):
            for s in (1, 2, 4):
                st, c = pgk.select_case_regs(m, TABLES["small"], 256, 256, 256, pgk.F32,
                                             pgk.params(b0, b1, s))
                if b0 <= b1 * s:
                    assert st == 0 and c.leaf == pgk.LEAF_4A3A and c.params.tile == b0
                else:
                    assert st == 2


def test_tensor_core_case_selection(built):
    """Tensor-core programs (host code): every default candidate of each form,
    CTA-pair programs (B0 = 256) included, selects its variant on a GB300-like
    machine; programs without a compiled variant are UNSUPPORTED, and a machine
    whose opt-in shared memory or compute capability does not fit makes a variant
    INFEASIBLE (its resource counters against the machine parameters)."""
    m = pgk.Machine(1024, 49152, 232448, 65536, 65536, 255, 2048, 152, 32, 10, 3, 0)
    for form in (pgk.BF16, pgk.SPLIT_BF16, pgk.FP8_E4M3):
        cands = pgk.default_candidates(form)
        assert cands
        for p in cands:
            # B1 = 64: the fused-conversion program, whose one tile covers N <= 64
            N = 64 if p.B1 == 64 else 8192
            st, c = pgk.select_case(m, 8192, N, 8192, form, p, raise_on_error=False)
            assert st == 0, (form, p.as_tuple(), pgk.last_error())
            assert (c.params.B0, c.params.B1, c.params.s) == (p.B0, p.B1, p.s)
            assert c.smem_bytes <= m.smem_per_block_optin and c.threads <= m.max_threads_per_block
            if p.B1 == 64:
                st, _ = pgk.select_case(m, 8192, 65, 8192, form, p, raise_on_error=False)
                assert st == 2, (form, p.as_tuple())
        for bad in [(256, 128, 3), (512, 256, 3), (128, 192, 4)]:
            st, _ = pgk.select_case(m, 8192, 8192, 8192, form, pgk.params(*bad, 0, 0),
                                    raise_on_error=False)
            assert st == 3, (form, bad)
    # K slices of the fused-conversion program (0: chosen at launch): kept in the case, bounded
    st, c = pgk.select_case(m, 4096, 16, 65536, pgk.SPLIT_BF16, pgk.params(128, 64, 3, 4, 0),
                            raise_on_error=False)
    assert st == 0 and c.params.sr == 4
    st, _ = pgk.select_case(m, 4096, 16, 65536, pgk.SPLIT_BF16, pgk.params(128, 64, 3, 5000, 0),
                            raise_on_error=False)
    assert st == 1
    # the fused-conversion program exists for BF16 and split, not for FP8
    assert any(p.B1 == 64 for p in pgk.default_candidates(pgk.SPLIT_BF16))
    assert any(p.B1 == 64 for p in pgk.default_candidates(pgk.BF16))
    assert not any(p.B1 == 64 for p in pgk.default_candidates(pgk.FP8_E4M3))
    # CTA pairs exist for the kind::f16 forms only
    assert any(p.B0 == 256 for p in pgk.default_candidates(pgk.SPLIT_BF16))
    assert any(p.B0 == 256 for p in pgk.default_candidates(pgk.BF16))
    st, _ = pgk.select_case(m, 8192, 8192, 8192, pgk.FP8_E4M3, pgk.params(256, 256, 6, 0, 0),
                            raise_on_error=False)
    assert st == 3
    small = pgk.Machine(1024, 49152, 200000, 65536, 65536, 255, 2048, 152, 32, 10, 3, 0)
    st, _ = pgk.select_case(small, 8192, 8192, 8192, pgk.SPLIT_BF16, pgk.params(256, 256, 3, 0, 0),
                            raise_on_error=False)
    assert st == 2
    hopper = pgk.Machine(1024, 49152, 232448, 65536, 65536, 255, 2048, 132, 32, 9, 0, 0)
    st, _ = pgk.select_case(hopper, 8192, 8192, 8192, pgk.BF16, pgk.params(128, 256, 4, 0, 0),
                            raise_on_error=False)
    assert st == 2
