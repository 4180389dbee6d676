// The case discussion at one concrete point (Algorithm 2 of Section 3).
//
// Resource counters, in their evaluation order r_1..r_4: threads per block (T),
// registers per thread (R), register file per block (R_B), shared memory per
// block (Z_B).  Strategies, in the order they are tried: "1" reduce register
// pressure (a register-capped build), "3b" reduce thread granularity,
// "4b" do not cache in shared memory.  sigma(registers) = {1},
// sigma(shared memory) = {3b, 4b}; the thread count has no strategy.
//
// At a concrete point exactly one of the accept (0 <= v <= R_i) and refuse
// (R_i < v) branches holds, so the walk follows that branch: accept moves to
// the next counter; refuse applies the first strategy of omega in sigma(r_i),
// removes it from omega and pushes r_1..r_i back on the counter stack (Remark
// "stacks": r_i ends on top); with no such strategy the branch is dropped and
// the point has no case.
//
// A Spec supplies the program state and the evaluation functions:
//   struct Spec {
//       struct Prog { ... };
//       pgk_status eval(int counter, const Prog&, long long* v);   // f_i
//       void apply(int strategy, Prog&);                            // O_j
//   };
#pragma once

#include "pgk_internal.cuh"

namespace pgk {

enum { C_THREADS = 0, C_REGS = 1, C_REGALLOC = 2, C_SMEM = 3, N_COUNTERS = 4 };
enum { O_REG = 0, O_GRAN = 1, O_NOCACHE = 2, N_STRATEGIES = 3 };

inline bool counter_in_sigma(int counter, int strategy) {
    switch (counter) {
        case C_REGS:
        case C_REGALLOC: return strategy == O_REG;
        case C_SMEM: return strategy == O_GRAN || strategy == O_NOCACHE;
        default: return false;
    }
}

inline long long counter_limit(int c, const pgk_machine& m) {
    switch (c) {
        case C_THREADS: return m.max_threads_per_block;
        case C_REGS: return m.max_regs_per_thread;
        case C_REGALLOC: return m.regs_per_block;
        default: return m.smem_per_block_optin;
    }
}

// Register file a block of `threads` needs: whole warps, 256-register units.
inline long long regalloc_bytes(long long threads, long long regs) {
    return ((threads + 31) / 32) * (((regs * 32) + 255) / 256 * 256);
}

template <class Spec>
pgk_status walk_cases(const pgk_machine& m, Spec& spec, typename Spec::Prog& p) {
    bool omega[N_STRATEGIES] = {true, true, true};
    int gamma[64];
    int top = 0;
    for (int c = N_COUNTERS - 1; c >= 0; --c) gamma[top++] = c;  // r_1 on top
    int guard = 0;
    while (top > 0) {
        if (++guard > 1000) {
            set_error("case walk did not terminate");
            return PGK_ERR_INFEASIBLE;
        }
        const int c = gamma[--top];
        long long v = 0;
        pgk_status st = spec.eval(c, p, &v);
        if (st != PGK_OK) return st;
        if (v >= 0 && v <= counter_limit(c, m)) continue;  // accept branch
        int chosen = -1;
        for (int o = 0; o < N_STRATEGIES; ++o)
            if (omega[o] && counter_in_sigma(c, o)) {
                chosen = o;
                break;
            }
        if (chosen < 0) {
            static const char* names[] = {"threads per block", "registers per thread",
                                          "register file per block", "shared memory per block"};
            set_error("no case: %s = %lld exceeds %lld and no strategy is left", names[c], v,
                      counter_limit(c, m));
            return PGK_ERR_INFEASIBLE;
        }
        spec.apply(chosen, p);
        omega[chosen] = false;
        for (int r = 0; r <= c; ++r) gamma[top++] = r;  // push r_1..r_i: r_i ends on top
    }
    return PGK_OK;
}

}  // namespace pgk
