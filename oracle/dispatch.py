"""Case-discussion oracle for the FP32 SIMT GEMM family -- TEST INFRASTRUCTURE ONLY.

Instantiates Algorithms 1 and 2 (module `comprehensive`) with the counters and
strategies of the parametric GEMM kernel of Fig. "cudamul" (Section 2), as the
paper's experiments do (Section 5): resource counters are the registers per
thread and the shared memory per block (plus the thread-block size and the
register file per block, the other two limits a launch on this GPU checks), no
performance counters, and the strategies

  "1"  reduce register pressure (applied to the IR: a register-capped build),
  "3b" reduce thread granularity (s -> 1),
  "4b" do not cache in shared memory,

tried in that order (omega = 1, 3b, 4b).  Leaves therefore carry the paper's
case labels (4a,3a), (3b,4a) and (3b,4b), each with or without "1".

Program state (the stand-in for the source CFG):
  family  "paper": each thread computes s outputs strided by B1; shared tiles
                   A: B0 x BK and B: BK x (B1 s)   (Fig. "cudamul" with BK = B0)
          "rb"   : register-blocked extension, sr x s outputs per thread in
                   float4 groups; double-buffered tiles A^T: BK x (B0 sr + 4)
                   and B: BK x (B1 s + 4)
          "direct": no shared memory, one output per thread
  s, sr, regopt.

Machine symbols: T (max threads per block), R (max registers per thread),
RB (registers per block), ZB (shared memory per block, bytes; the paper counts
words, Section 3.2).  Program symbols: B0, B1, s, sr, BK.
"""
from __future__ import annotations

from . import comprehensive as co

STRATEGY_ORDER = ["1", "3b", "4b"]


def smem_bytes_formula(prog: dict):
    """f_smem on the source: bytes of shared memory one block allocates."""
    fam = prog["family"]
    if not prog["cache"] or fam == "direct":
        return "0", lambda e: 0 * e["B0"]
    if fam == "paper":
        s = prog["s"]
        if s == "s":
            return "4(B0 BK + BK B1 s)", lambda e: 4 * (e["B0"] * e["BK"] + e["BK"] * e["B1"] * e["s"])
        return f"4(B0 BK + BK B1 {s})", lambda e, s=s: 4 * (e["B0"] * e["BK"] + e["BK"] * e["B1"] * s)
    # register-blocked: two buffers of A^T (BK x (B0 sr + 4)) and B (BK x (B1 s + 4))
    return ("8 BK (B0 sr + B1 s + 8)",
            lambda e: 8 * e["BK"] * (e["B0"] * e["sr"] + e["B1"] * e["s"] + 8))


def make_counters(regs_of):
    """`regs_of(prog)` returns a function env -> registers per thread of the
    variant `prog` (the IR evaluation function f_regs of step S2)."""

    def ev_threads(prog):
        return "B0 B1", lambda e: e["B0"] * e["B1"]

    def ev_regs(prog):
        return f"regs{_tag(prog)}", regs_of(prog)

    def ev_regalloc(prog):
        r = regs_of(prog)

        def v(e):
            warps = (e["B0"] * e["B1"] + 31) // 32
            return warps * (((r(e) * 32) + 255) // 256 * 256)
        return f"ceil(B0 B1/32) roundup(32 regs{_tag(prog)}, 256)", v

    return {
        "r_threads": co.Counter("r_threads", "resource", "T", ev_threads, ()),
        "r_regs": co.Counter("r_regs", "resource", "R", ev_regs, ("1",)),
        "r_regalloc": co.Counter("r_regalloc", "resource", "RB", ev_regalloc, ("1",)),
        "r_smem": co.Counter("r_smem", "resource", "ZB", smem_bytes_formula, ("3b", "4b")),
    }


def _tag(prog):
    return f"[{prog['family']},s={prog['s']},sr={prog['sr']},cap={int(prog['regopt'])}]"


def _o_reg(p):
    p = dict(p)
    p["regopt"] = True
    return p


def _o_gran(p):
    p = dict(p)
    p["s"] = 1
    p["sr"] = 1
    if p["family"] == "rb":
        p["family"] = "paper"
    return p


def _o_nocache(p):
    p = dict(p)
    p["cache"] = False
    p["family"] = "direct"
    return p


STRATEGIES = {
    "1": co.Strategy("1", True, _o_reg),
    "3b": co.Strategy("3b", False, _o_gran),
    "4b": co.Strategy("4b", False, _o_nocache),
}


def initial_program(family: str) -> dict:
    return {"family": family, "cache": True, "s": "s", "sr": "sr" if family == "rb" else 1,
            "regopt": False}


def precondition():
    """Initial constraints C(S): parameters positive, and the assertion of
    Fig. "metamul", B0 <= ub1 * s (here B1 plays ub1)."""
    return [co.Constraint("B0 >= 1, B1 >= 1, s >= 1, BK >= 1",
                          lambda e: (e["B0"] >= 1) & (e["B1"] >= 1) & (e["s"] >= 1) & (e["BK"] >= 1)),
            co.Constraint("B0 <= B1 s", lambda e: e["B0"] <= e["B1"] * e["s"])]


def case_tree(family: str, regs_of, box):
    counters = make_counters(regs_of)
    Q = co.initial_quintuple(initial_program(family), STRATEGY_ORDER,
                             ["r_threads", "r_regs", "r_regalloc", "r_smem"], precondition())
    return co.comprehensive_optimization(Q, counters, STRATEGIES, box)


def leaf_label(prog: dict, lam: list) -> str:
    """The paper's decision labels (Section 5): "(1)" when no register-pressure
    optimisation was applied, (4a)/(4b) cache or not, (3a)/(3b) granularity kept
    or reduced."""
    reg = "(1)" if "1" not in lam else "(reg)"
    cache = "(4a)" if prog["cache"] else "(4b)"
    gran = "(3a)" if prog["s"] == "s" else "(3b)"
    return reg + cache + gran


def leaf_code(prog: dict) -> int:
    """Library leaf numbering: 0 = (4a,3a), 1 = (3b,4a), 2 = (3b,4b)."""
    if not prog["cache"]:
        return 2
    return 0 if prog["s"] == "s" else 1


def brute_force(leaves, env):
    """Evaluate every leaf's conjunction separately at the points of `env`.
    Returns, per point, the list of leaf indices whose system holds."""
    import numpy as np
    n = len(next(iter(env.values())))
    hits = [[] for _ in range(n)]
    for li, (_, _, C) in enumerate(leaves):
        ok = co.holds(C, env)
        for idx in np.nonzero(ok)[0]:
            hits[idx].append(li)
    return hits


# ----------------------------------------------- transposition and 1D Jacobi
# The same counters and strategies for the paper's two other kernels, with the
# shared-memory formulas of their GB300 variants:
#   transposition: the a tile of B0 rows x (B1 s + 1) words, 4 B0 (B1 s + 1) bytes;
#   Jacobi: read window s B + 2 words and s B results, 4 (2 s B + 2) bytes
#   (Fig. "1dj" counts 2 s B + 2 words).
# There is no register-capped build of these kernels, so strategy "1" leaves the
# register count unchanged.

def stencil_counters(kind, regs_of):
    def ev_threads(prog):
        if kind == "transpose":
            return "B0 B1", lambda e: e["B0"] * e["B1"]
        return "B", lambda e: e["B0"]

    def ev_regs(prog):
        return "regs", regs_of(prog)

    def ev_regalloc(prog):
        r = regs_of(prog)
        th = ev_threads(prog)[1]

        def v(e):
            return (th(e) + 31) // 32 * (((r(e) * 32) + 255) // 256 * 256)
        return "regalloc", v

    def ev_smem(prog):
        if not prog["cache"]:
            return "0", lambda e: 0 * e["B0"]
        if kind == "transpose":
            if prog["s"] == "s":
                return "4 B0 (B1 s + 1)", lambda e: 4 * e["B0"] * (e["B1"] * e["s"] + 1)
            return "4 B0 (B1 + 1)", lambda e: 4 * e["B0"] * (e["B1"] + 1)
        if prog["s"] == "s":
            return "4 (2 s B + 2)", lambda e: 4 * (2 * e["s"] * e["B0"] + 2)
        return "4 (2 B + 2)", lambda e: 4 * (2 * e["B0"] + 2)

    return {
        "r_threads": co.Counter("r_threads", "resource", "T", ev_threads, ()),
        "r_regs": co.Counter("r_regs", "resource", "R", ev_regs, ("1",)),
        "r_regalloc": co.Counter("r_regalloc", "resource", "RB", ev_regalloc, ("1",)),
        "r_smem": co.Counter("r_smem", "resource", "ZB", ev_smem, ("3b", "4b")),
    }


STENCIL_STRATEGIES = {
    "1": co.Strategy("1", True, lambda p: dict(p, regopt=True)),
    "3b": co.Strategy("3b", False, lambda p: dict(p, s=1)),
    "4b": co.Strategy("4b", False, lambda p: dict(p, cache=False)),
}


def stencil_case_tree(kind, regs_of, box):
    Q = co.initial_quintuple({"cache": True, "s": "s", "regopt": False}, STRATEGY_ORDER,
                             ["r_threads", "r_regs", "r_regalloc", "r_smem"],
                             [co.Constraint("B0, B1, s >= 1",
                                            lambda e: (e["B0"] >= 1) & (e["B1"] >= 1) & (e["s"] >= 1))])
    return co.comprehensive_optimization(Q, stencil_counters(kind, regs_of), STENCIL_STRATEGIES, box)
