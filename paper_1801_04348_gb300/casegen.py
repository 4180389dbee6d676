"""Offline case-table generator: Algorithms 1 and 2 of the paper (Section 3)
applied to a kernel description, emitting the comprehensive parametric kernel as
a list of (constraint system, optimised program) pairs, the form of Fig.
"compparkern" and of the case systems printed in Section 5.

The quintuple Q(S) = (program, lambda, omega, gamma, C) is processed with an
explicit work list instead of recursion: popping a node takes the next counter c
off gamma and evaluates it; the accept child adds 0 <= v <= R_c; the refuse
child adds R_c < v, applies the first strategy of omega that belongs to
sigma(c), and pushes r_1..r_c back on gamma (r_c on top, Remark "stacks").
Children whose system has no solution are discarded; the consistency of a
system is decided by enumerating a finite box of non-negative integer points
(hypothesis H1) in place of RealTriangularize.  Nodes with an empty gamma are
the leaves.

    python -m paper_1801_04348_gb300.casegen --kernel gemm --machine m2050

prints the GEMM family's case table for a Fermi-like machine (registers from a
mock table); `--machine current` reads the machine and the compiled variants'
registers from the GPU.
"""
from __future__ import annotations

import argparse
import json
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Counter:
    name: str
    limit: str                       # machine parameter symbol
    sigma: tuple                     # strategies that may reduce it
    value: object                    # (prog, env) -> numpy array
    text: object                     # prog -> printable expression


@dataclass
class Strategy:
    label: str                       # the paper's decision label
    on_ir: bool
    apply: object                    # prog -> prog


@dataclass
class Node:
    prog: dict
    lam: tuple = ()
    omega: tuple = ()
    gamma: tuple = ()
    system: tuple = ()               # ((text, mask), ...)
    labels: tuple = ()


@dataclass
class KernelSpec:
    name: str
    program: dict
    counters: list                   # in the order r_1, r_2, ...
    strategies: list                 # omega's initial order
    precondition: list = field(default_factory=list)   # [(text, env -> mask)]


def make_box(ranges: dict) -> dict:
    names = list(ranges)
    grids = np.meshgrid(*[np.asarray(list(ranges[n]), dtype=np.int64) for n in names], indexing="ij")
    return {n: g.reshape(-1) for n, g in zip(names, grids)}


def generate(spec: KernelSpec, box: dict) -> list:
    """Leaves of the tree T(Q(S)): processed nodes with consistent systems."""
    npts = len(next(iter(box.values())))
    mask0 = np.ones(npts, dtype=bool)
    pre = []
    for text, pred in spec.precondition:
        m = np.asarray(pred(box), dtype=bool)
        mask0 &= m
        pre.append((text, m))
    counters = {c.name: c for c in spec.counters}
    order = [c.name for c in spec.counters]
    root = Node(prog=dict(spec.program), omega=tuple(s.label for s in spec.strategies),
                gamma=tuple(order), system=tuple(pre))
    strategies = {s.label: s for s in spec.strategies}
    work = [(root, mask0)]
    leaves = []
    while work:
        node, mask = work.pop()
        if not node.gamma:
            leaves.append((node, mask))
            continue
        c = counters[node.gamma[0]]
        rest = node.gamma[1:]
        v = np.asarray(c.value(node.prog, box))
        lim = box[c.limit]
        ok = (v >= 0) & (v <= lim)
        acc_mask = mask & ok
        if acc_mask.any():
            work.append((Node(node.prog, node.lam, node.omega, rest,
                              node.system + ((f"0 <= {c.text(node.prog)} <= {c.limit}", ok),),
                              node.labels), acc_mask))
        ref = lim < v
        ref_mask = mask & ref
        chosen = next((o for o in node.omega if o in c.sigma), None)
        if chosen is None or not ref_mask.any():
            continue
        st = strategies[chosen]
        i = order.index(c.name)
        requeue = tuple(reversed(order[: i + 1]))       # r_i on top, then r_{i-1} .. r_1
        work.append((Node(st.apply(dict(node.prog)),
                          node.lam + ((chosen,) if st.on_ir else ()),
                          tuple(o for o in node.omega if o != chosen),
                          requeue + rest,
                          node.system + ((f"{c.limit} < {c.text(node.prog)}", ref),),
                          node.labels + (chosen,)), ref_mask))
    return leaves


def leaf_region(leaves, pick) -> np.ndarray:
    """Union of the masks of the leaves whose program satisfies `pick`."""
    out = None
    for node, mask in leaves:
        if pick(node.prog):
            out = mask.copy() if out is None else (out | mask)
    return out


def table_text(spec: KernelSpec, leaves) -> str:
    lines = [f"comprehensive parametric kernel: {spec.name} ({len(leaves)} cases)"]
    for k, (node, mask) in enumerate(leaves, 1):
        lab = " ".join(f"({l})" for l in node.labels) or "(none)"
        lines.append(f"case {k}: strategies {lab}; program {node.prog}; {int(mask.sum())} box points")
        for text, _ in node.system:
            lines.append(f"    {text}")
    return "\n".join(lines)


# --------------------------------------------------------------- kernels
def _regalloc(threads, regs):
    return (threads + 31) // 32 * (((regs * 32) + 255) // 256 * 256)


def gemm_spec(regs_table) -> KernelSpec:
    """The FP32 SIMT GEMM family (Fig. "cudamul"): paper-form (sr = 1) programs.
    regs_table: the PGK_REG_CLASSES register counts (paper s = 1, 2, 4, 8; capped;
    direct; direct capped; register-blocked)."""
    sidx = {1: 0, 2: 1, 4: 2, 8: 3}

    def regs(p, e):
        if not p["cache"]:
            return np.full_like(e["B0"], regs_table[9 if p["cap"] else 8])
        base = 4 if p["cap"] else 0
        if p["s"] == "s":
            out = np.zeros_like(e["s"])
            for sv, si in sidx.items():
                out = np.where(e["s"] == sv, regs_table[base + si], out)
            return out
        return np.full_like(e["B0"], regs_table[base + sidx[p["s"]]])

    def smem(p, e):
        if not p["cache"]:
            return 0 * e["B0"]
        s = e["s"] if p["s"] == "s" else p["s"]
        return 4 * (e["B0"] * e["BK"] + e["BK"] * e["B1"] * s)

    def gran(p):
        p["s"] = 1
        return p

    def nocache(p):
        p["cache"] = False
        return p

    def cap(p):
        p["cap"] = True
        return p

    tag = lambda p: f"[s={p['s']},{'cache' if p['cache'] else 'direct'}{',capped' if p['cap'] else ''}]"
    return KernelSpec(
        "GEMM (paper form)", {"s": "s", "cache": True, "cap": False},
        [Counter("threads", "T", (), lambda p, e: e["B0"] * e["B1"], lambda p: "B0*B1"),
         Counter("regs", "R", ("1",), regs, lambda p: f"regs{tag(p)}"),
         Counter("regfile", "RB", ("1",), lambda p, e: _regalloc(e["B0"] * e["B1"], regs(p, e)),
                 lambda p: f"warps*roundup(32*regs{tag(p)},256)"),
         Counter("smem", "ZB", ("3b", "4b"), smem,
                 lambda p: "0" if not p["cache"] else f"4*(B0*BK + BK*B1*{p['s']})")],
        [Strategy("1", True, cap), Strategy("3b", False, gran), Strategy("4b", False, nocache)],
        [("B0 <= B1*s", lambda e: e["B0"] <= e["B1"] * e["s"])])


def matrix_add_spec() -> KernelSpec:
    """Fig. "compparkern": registers 14, 10 after reducing granularity."""
    return KernelSpec(
        "matrix addition (Fig. compparkern)", {"kernel": "K1", "regs": 14},
        [Counter("threads", "T", (), lambda p, e: e["B0"] * e["B1"], lambda p: "B0*B1"),
         Counter("regs", "R", ("3b",), lambda p, e: np.full_like(e["R"], p["regs"]),
                 lambda p: str(p["regs"]))],
        [Strategy("3b", False, lambda p: {"kernel": "K2", "regs": 10})])


MACHINES = {
    # Fermi-like (public M2050 specifications, not from the paper)
    "m2050": {"T": [1024], "R": [63], "RB": [32768], "ZB": [49152]},
    # a small machine that forces the (3b,4a) and (3b,4b) leaves
    "tiny": {"T": [512], "R": [63], "RB": [16384], "ZB": [1024, 2048, 4096]},
}


def main():
    ap = argparse.ArgumentParser(description="emit a comprehensive parametric kernel (case table)")
    ap.add_argument("--kernel", default="gemm", choices=["gemm", "matrix_add"])
    ap.add_argument("--machine", default="m2050", choices=["m2050", "tiny", "current"])
    ap.add_argument("--json", action="store_true")
    args = ap.parse_args()
    if args.kernel == "matrix_add":
        spec = matrix_add_spec()
        box = make_box({"R": range(0, 64), "T": [256, 512, 1024], "B0": [1, 2, 4, 8, 16, 32],
                        "B1": [1, 2, 4, 8, 16, 32]})
    else:
        if args.machine == "current":
            from . import pgk
            m = pgk.machine_query(0)
            mach = {"T": [m.max_threads_per_block], "R": [m.max_regs_per_thread],
                    "RB": [m.regs_per_block], "ZB": [m.smem_per_block_optin]}
            regs = []
            for fam, s, cap in [(pgk.FAM_PAPER, s, c) for c in (0, 1) for s in (1, 2, 4, 8)] + \
                               [(pgk.FAM_DIRECT, 1, 0), (pgk.FAM_DIRECT, 1, 1), (pgk.FAM_RB, 0, 0)]:
                r = 0
                for i in range(pgk.num_variants()):
                    v = pgk.variant_info_get(i)
                    if v.family == fam and (fam == pgk.FAM_RB or (v.s == s and v.regopt == cap)):
                        r = v.regs
                        break
                regs.append(r)
        else:
            mach = MACHINES[args.machine]
            regs = [30, 34, 40, 56, 30, 32, 32, 40, 24, 24, 128]
        spec = gemm_spec(regs)
        box = make_box(dict(mach, B0=[8, 16, 32], B1=[8, 16, 32], s=[1, 2, 4], BK=[8, 16, 32]))
    leaves = generate(spec, box)
    if args.json:
        print(json.dumps([{"strategies": n.labels, "ir_strategies": n.lam, "program": n.prog,
                           "system": [t for t, _ in n.system], "points": int(m.sum())}
                          for n, m in leaves]))
    else:
        print(table_text(spec, leaves))


if __name__ == "__main__":
    main()
