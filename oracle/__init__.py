"""CPU oracle for the parametric GEMM kernel family -- TEST INFRASTRUCTURE ONLY.

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import anything from this package.  It shares no code with the CUDA path
(`paper_1801_04348_gb300`), and that package never imports it.

Modules:
  gemm           FP64 definition C = beta*C0 + A*B (plain C, OpenMP), long-double self-check,
                 int32 modulo 2^32 form (the paper's data type)
  quant          BF16 / FP8-E4M3 / split-BF16 / per-tile FP8 scaling from the format definitions
  mlp            FP64 forward, backward and Adam step of the 7-64-64-1 cost model
  comprehensive  Algorithms 1 and 2 of the paper (comprehensive optimization)
  dispatch       the GEMM family's counters and strategies, brute-force case evaluation
"""
from .gemm import build, gemm, gemm_i32, gemm_longdouble, max_threads, rel_frobenius  # noqa: F401
