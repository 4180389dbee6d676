"""Comprehensive optimization (Algorithms 1 and 2, Section 3) -- TEST INFRASTRUCTURE ONLY.

A direct, unoptimised restatement of the paper's procedure, used as the oracle
for the library's case dispatcher:

* A quintuple Q(S) = (G_C(S), lambda(S), omega(S), gamma(S), C(S)) (Section 3.5):
  the program (here a small dict of variant choices standing in for the CFG),
  the strategies already applied to the IR, the strategies not yet applied, the
  counters still to evaluate, and the constraint system built so far.  The four
  sequences are stacks with the push/pop conventions of Remark "stacks".
* Optimize (Algorithm 2) pops the next counter c, evaluates it on the program,
  forks an accept branch (0 <= v <= R_i, resp. 0 <= v <= P_i) and a refuse
  branch (R_i < v, resp. P_i < v <= 1); the refuse branch applies the first
  strategy of omega that belongs to sigma(c), pushes the counters r_1..r_i
  (resp. r_1..r_s, p_i) back onto gamma and recurses; with no such strategy the
  refuse branch is dropped.  Inconsistent systems are removed.
* ComprehensiveOptimization (Algorithm 1) recurses until gamma is empty and
  returns the processed (program, lambda, C) triples.

The paper decides consistency with RealTriangularize (RegularChains/Maple).  This
oracle decides it by enumeration over a finite box of integer points (all
parameters are non-negative integers, hypothesis H1): a system is consistent iff
at least one point of the box satisfies every constraint.  Constraints are
predicates evaluated on numpy arrays holding every point of the box at once.
"""
from __future__ import annotations

import copy
import itertools
from dataclasses import dataclass, field
from typing import Callable

import numpy as np

Env = dict  # symbol -> numpy array (one entry per point of the box)


@dataclass
class Constraint:
    text: str
    pred: Callable[[Env], np.ndarray]


@dataclass
class Counter:
    """A resource counter r_i (kind 'resource', bounded by machine parameter
    `limit`) or a performance counter p_i (kind 'performance', a ratio that the
    machine parameter `limit` caps).  `evaluate(program)` is the evaluation
    function f_i / g_i: it returns (printable text, function env -> values)."""
    name: str
    kind: str
    limit: str
    evaluate: Callable[[dict], tuple]
    sigma: tuple = ()


@dataclass
class Strategy:
    name: str
    on_ir: bool
    apply: Callable[[dict], dict]


@dataclass
class Quintuple:
    program: dict
    lam: list = field(default_factory=list)     # applied IR strategies
    omega: list = field(default_factory=list)   # strategies not yet applied
    gamma: list = field(default_factory=list)   # counters left to evaluate (stack)
    C: list = field(default_factory=list)       # constraint system


def initial_quintuple(program: dict, strategies: list, counters: list,
                      constraints: list) -> Quintuple:
    """lambda empty, omega = O_1..O_w, gamma = r_1..r_s, p_1..p_t (r_1 on top)."""
    return Quintuple(program=dict(program), lam=[], omega=list(strategies),
                     gamma=list(counters), C=list(constraints))


def push_sequence(stack: list, seq: list) -> None:
    """Remark "stacks": pushing t_1..t_M on s_1..s_N gives t_M..t_1, s_1..s_N
    (index 0 is the top)."""
    for t in seq:
        stack.insert(0, t)


def consistent(C: list, box: Env) -> bool:
    if not C:
        return True
    n = len(next(iter(box.values())))
    ok = np.ones(n, dtype=bool)
    for c in C:
        ok &= np.asarray(c.pred(box), dtype=bool)
        if not ok.any():
            return False
    return True


def optimize(Q: Quintuple, counters: dict, strategies: dict, box: Env) -> list:
    """Algorithm 2.  Returns a list of quintuples (the stack `result`)."""
    result = []
    cname = Q.gamma.pop(0)
    c = counters[cname]
    text, v = c.evaluate(Q.program)
    lim = c.limit
    Q2 = copy.deepcopy(Q)                               # refuse branch copy
    if c.kind == "resource":
        Q.C.append(Constraint(f"0 <= {text} <= {lim}",
                              lambda e, v=v, lim=lim: (v(e) >= 0) & (v(e) <= e[lim])))
        result.insert(0, Q)
        Q2.C.append(Constraint(f"{lim} < {text}", lambda e, v=v, lim=lim: e[lim] < v(e)))
        requeue = [k for k in _resource_names(counters)]
        requeue = requeue[: requeue.index(cname) + 1]    # r_1 .. r_i
    else:
        Q.C.append(Constraint(f"0 <= {text} <= {lim}",
                              lambda e, v=v, lim=lim: (v(e) >= 0) & (v(e) <= e[lim])))
        result.insert(0, Q)
        Q2.C.append(Constraint(f"{lim} < {text} <= 1",
                               lambda e, v=v, lim=lim: (e[lim] < v(e)) & (v(e) <= 1)))
        requeue = _resource_names(counters) + [cname]    # r_1 .. r_s, p_i
    chosen = next((s for s in Q2.omega if s in c.sigma), None)
    if chosen is not None:
        st = strategies[chosen]
        Q3 = Q2
        Q3.program = st.apply(dict(Q3.program))
        Q3.omega = [s for s in Q3.omega if s != chosen]
        if st.on_ir:
            Q3.lam.append(chosen)
        push_sequence(Q3.gamma, requeue)
        for q in optimize(Q3, counters, strategies, box):
            result.insert(0, q)
    return [q for q in result if consistent(q.C, box)]


def _resource_names(counters: dict) -> list:
    return [k for k, c in counters.items() if c.kind == "resource"]


def comprehensive_optimization(Q: Quintuple, counters: dict, strategies: dict,
                               box: Env) -> list:
    """Algorithm 1.  Returns the processed triples (program, lambda, C)."""
    if not Q.gamma:
        return [(Q.program, list(Q.lam), list(Q.C))]
    out = []
    for Qp in optimize(Q, counters, strategies, box):
        out = comprehensive_optimization(Qp, counters, strategies, box) + out
    return out


def tree_height_bound(n_strategies: int, n_resource: int, n_perf: int) -> int:
    """Lemma 1: the height of the tree T(Q(S)) is at most w (s + t)."""
    return n_strategies * (n_resource + n_perf)


def make_box(ranges: dict) -> Env:
    """Cartesian product of integer ranges, as one flat array per symbol."""
    names = list(ranges)
    grids = np.meshgrid(*[np.asarray(list(ranges[n]), dtype=np.int64) for n in names],
                        indexing="ij")
    return {n: g.reshape(-1) for n, g in zip(names, grids)}


def holds(C: list, env: Env) -> np.ndarray:
    n = len(next(iter(env.values())))
    ok = np.ones(n, dtype=bool)
    for c in C:
        ok &= np.asarray(c.pred(env), dtype=bool)
    return ok


def point_env(point: dict) -> Env:
    return {k: np.asarray([v], dtype=np.int64) for k, v in point.items()}


def all_points(ranges: dict):
    names = list(ranges)
    for vals in itertools.product(*[list(ranges[n]) for n in names]):
        yield dict(zip(names, vals))
