"""Measurements of the GEMM workloads beside the headline benchmark.

    python experiments.py --out DIR [config1 scale grouped precision ...]

config1    M = N = K = 256, uniform[-1,1] seed 0: every (B0, B1, s) of {8,16,32}^2 x {1,2,4};
           case leaf, registers, time, and relative error against an FP64 product.
scale      FP32 at 4096^3, 8192^3, 8192 x 1024 x 4096, 16384 x 64 x 16384: full autotune
           sweep of the register-blocked variants, best time, TFLOP/s, fraction of the SIMT
           peak (152 SMs x 128 lanes x 2 flop x 2070 MHz), and GB/s of compulsory traffic.
grouped    512 FP32 GEMMs, M, N, K log-uniform in [32, 2048] (multiples of 16, seed 0),
           normal(0,1) operands: one grouped persistent launch (eager and CUDA-graph
           replay, tile variant from pgk_autotune_grouped) against 512 separate pgk_gemm
           launches (eager and captured in one CUDA graph); and the same group in the
           BF16 and split forms (grouped conversions + one tensor-core launch).
mm         the paper's Table "mm" grid on GB300: int32, n = 2^10 and 2^11, (ub1, B0) x s.
transpose  the paper's transposition grid at order 2^14 (GB/s).
jacobi     the paper's 1D Jacobi grid (T = 4, length 2^15 + 2; and 2^27 + 2).
errmeas    the FP64 error reduction on 8192^2 (GB/s).
mlp        the cost-model kernels (forward, minibatch gradient + Adam, full gradient).
forms      every form (FP32, BF16, split, FP8) at 4096^3, 8192 x 1024 x 4096 and
           16384 x 64 x 16384: step and kernel time, error on 64 sampled rows.
link       the host link with pinned buffers (256 MiB copies: host-to-device, device-to-host,
           both at once) and the end-to-end step of pgk_gemm_host at 8192^3 (split form).
peaks      the library's FP32 FMA probe (paired and scalar) with the SM clock during it,
           and, as context only, PyTorch's BF16 matmul and FP8 scaled matmul at 8192^3.
precision  8192^3, normal(0,1) and row-scaled by 10^uniform(-3,3): every form's step
           time (FP32 in/out, preparation included), kernel time on prepared operands,
           and relative Frobenius error on 64 sampled rows against an FP64 product.

--only B0,B1,s[,sr,tile] restricts mm (n = 2^11), transpose and jacobi (2^27 + 2 points) to
one program point, for profiling a single kernel.

Timing: CUDA events on the launching stream after warm-up; medians of repeated runs.
Error columns compare with numpy's binary64 product of the same FP32 operands on
sampled rows (a measurement reference; the parity tests under tests/ compare with
the oracle).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import time

import numpy as np

import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1801_04348_gb300 import inputs, pgk  # noqa: E402

PEAK_MHZ = 2070.0
ONLY = None   # --only B0,B1,s: run a single program point of mm / transpose / jacobi (profiling)


def _events_ms(fn, reps, stream):
    import torch
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def _ref_rows(A, B, rows):
    """Rows of the binary64 product of the FP32 operands (numpy)."""
    return A[rows].astype(np.float64) @ B.astype(np.float64)


def _rel_frob(got, ref):
    got = np.asarray(got, dtype=np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def _rel_err_rows(Cd, A, B, rows):
    import torch
    got = Cd[torch.from_numpy(rows).to(Cd.device)].cpu().numpy()
    return _rel_frob(got, _ref_rows(A, B, rows))


def simt_peak(machine):
    return machine.sm_count * 128 * 2 * PEAK_MHZ * 1e6 / 1e12


def config1(dev, stream):
    import torch
    M = N = K = 256
    A, B = inputs.gemm_operands(M, N, K, seed=0)
    Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    C = torch.empty(M, N, device=dev)
    m = pgk.machine_query(dev.index or 0)
    rows = np.arange(M, dtype=np.int64)
    out = []
    for b0 in (8, 16, 32):
        for b1 in (8, 16, 32):
            for s in (1, 2, 4):
                p = pgk.params(b0, b1, s)
                st, c = pgk.select_case(m, M, N, K, pgk.F32, p, raise_on_error=False)
                rec = {"B0": b0, "B1": b1, "s": s, "status": pgk.STATUS[st]}
                if st == 0:
                    run = lambda: pgk.gemm(Ad, Bd, C, pgk.F32, p, stream=stream)
                    run()
                    ms = _events_ms(run, 20, stream)
                    rec.update(leaf=c.leaf, regs=c.regs, smem=c.smem_bytes, ms=ms,
                               tflops=2.0 * M * N * K / ms / 1e9,
                               rel_err=_rel_err_rows(C, A, B, rows))
                out.append(rec)
    return {"config": "config1 256^3 paper-form grid", "points": out,
            "feasible": sum(1 for r in out if r["status"] == "PGK_OK")}


def scale(dev, stream):
    import torch
    m = pgk.machine_query(dev.index or 0)
    peak = simt_peak(m)
    res = []
    cands = [p for p in pgk.default_candidates(pgk.F32) if p.sr > 1]
    for (M, N, K) in [(4096, 4096, 4096), (8192, 8192, 8192), (8192, 1024, 4096), (16384, 64, 16384)]:
        A, B = inputs.gemm_operands(M, N, K, seed=0)
        Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
        C = torch.empty(M, N, device=dev)
        best, table = pgk.autotune(Ad, Bd, C, pgk.F32, candidates=cands, reps=3, stream=stream)
        run = lambda: pgk.gemm(Ad, Bd, C, pgk.F32, best, stream=stream)
        ms = _events_ms(run, 5, stream)
        rows = np.linspace(0, M - 1, 32).astype(np.int64)
        fl = 2.0 * M * N * K
        byt = 4.0 * (M * K + K * N + M * N)
        res.append({"M": M, "N": N, "K": K, "best": list(best.as_tuple()), "ms": ms,
                    "tflops": fl / ms / 1e9, "simt_peak_tflops": peak,
                    "frac_of_simt_peak": fl / ms / 1e9 / peak, "gbs": byt / ms / 1e6,
                    "rel_err_32_rows": _rel_err_rows(C, A, B, rows),
                    "sweep": [(list(p.as_tuple()), t) for p, t in table]})
        del Ad, Bd, C
        torch.cuda.empty_cache()
    return {"config": "scale FP32 tuned", "shapes": res}


def grouped(dev, stream):
    import torch
    dims = inputs.log_uniform_dims(512, 0, 32, 2048, 16)
    trip = []
    for i, (M, N, K) in enumerate(dims):
        A, B = inputs.gemm_operands(int(M), int(N), int(K), seed=1 + 2 * i, dist="normal")
        trip.append((torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev),
                     torch.empty(int(M), int(N), device=dev)))
    flops = float(sum(2.0 * int(M) * int(N) * int(K) for M, N, K in dims))
    probs = pgk.make_problems(trip)
    best, table = pgk.autotune_grouped(probs, reps=3, stream=stream)
    sh = stream.cuda_stream
    eager = lambda: pgk.gemm_grouped(probs, pgk.F32, best, stream=sh)
    graph = lambda: pgk.gemm_grouped(probs, pgk.F32, best, use_graph=1, stream=sh)
    eager()
    graph()
    t_grouped = _events_ms(eager, 10, stream)
    t_grouped_graph = _events_ms(graph, 10, stream)

    def separate():
        for A, B, C in trip:
            pgk.gemm(A, B, C, pgk.F32, None, stream=sh)
    separate()
    t_sep = _events_ms(separate, 5, stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        separate()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
            separate()
    replay = lambda: g.replay()
    replay()
    t_sep_graph = _events_ms(replay, 10, stream)
    # the tensor-core forms of the same group (BF16 and split: one conversion launch for
    # A and B, one GEMM launch; FP8: two quantisation launches and the GEMM)
    host_rows = []
    for i, (M, N, K) in enumerate(dims[:64]):
        A, B = inputs.gemm_operands(int(M), int(N), int(K), seed=1 + 2 * i, dist="normal")
        rows = np.unique(np.linspace(0, int(M) - 1, 4).astype(np.int64))
        host_rows.append((rows, _ref_rows(A, B, rows)))
    tc = {}
    for name, dt, prog in (("bf16", pgk.BF16, pgk.params(128, 128, 6, 0, 64)),
                           ("split", pgk.SPLIT_BF16, pgk.params(128, 128, 3, 0, 64)),
                           ("split3", pgk.SPLIT_BF16, pgk.params(128, 128, 6, 0, 64)),
                           ("fp8", pgk.FP8_E4M3, pgk.params(128, 128, 6, 0, 128))):
        run = lambda: pgk.gemm_grouped(probs, dt, prog, stream=sh)
        run()
        ms = _events_ms(run, 10, stream)
        torch.cuda.synchronize()
        err = max(_rel_frob(trip[i][2][torch.from_numpy(r).to(dev)].cpu().numpy(), ref)
                  for i, (r, ref) in enumerate(host_rows))
        tc[name] = {"params": list(prog.as_tuple()), "ms": ms, "tflops": flops / ms / 1e9,
                    "max_rel_err_first_64_problems": err}
    return {"config": "grouped 512 GEMMs", "flops": flops, "tile_variant": list(best.as_tuple()),
            "tensor_core_forms": tc,
            "variant_sweep_ms": [(list(p.as_tuple()), t) for p, t in table],
            "grouped_ms": t_grouped, "grouped_graph_ms": t_grouped_graph,
            "separate_ms": t_sep, "separate_graph_ms": t_sep_graph,
            "tflops": {"grouped": flops / t_grouped / 1e9,
                       "grouped_graph": flops / t_grouped_graph / 1e9,
                       "separate": flops / t_sep / 1e9,
                       "separate_graph": flops / t_sep_graph / 1e9}}


def _forms_at(M, N, K, dist, dev, stream):
    """Every form at one shape: autotuned program, step time (FP32 in / FP32 out,
    preparation included), kernel time on prepared operands, and the relative
    Frobenius error on 64 sampled rows against the binary64 product."""
    import torch
    sh = stream.cuda_stream
    out = []
    A, B = inputs.gemm_operands(M, N, K, seed=0, dist=dist)
    Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    C = torch.empty(M, N, device=dev)
    rows = np.linspace(0, M - 1, 64).astype(np.int64)
    for name, dt in (("f32", pgk.F32), ("bf16", pgk.BF16), ("split", pgk.SPLIT_BF16),
                     ("fp8", pgk.FP8_E4M3)):
        cands = [p for p in pgk.default_candidates(dt) if dt != pgk.F32 or p.sr > 1]
        best, _ = pgk.autotune(Ad, Bd, C, dt, candidates=cands, reps=2, stream=stream)
        run = lambda: pgk.gemm(Ad, Bd, C, dt, best, stream=sh)
        run()
        step_ms = _events_ms(run, 10, stream)
        err = _rel_err_rows(C, A, B, rows)
        kern_ms = step_ms
        pipe = 6.0 if dt == pgk.SPLIT_BF16 else 2.0
        # a fused-conversion program (B1 = 64) reads FP32 A itself: its call is the kernel
        if dt != pgk.F32 and best.B1 != 64:
            Kp = (K + 15) // 16 * 16
            if dt == pgk.FP8_E4M3:
                a = torch.empty(M, Kp, dtype=torch.uint8, device=dev)
                b = torch.empty(N, Kp, dtype=torch.uint8, device=dev)
                sa = torch.empty((M + 127) // 128, (K + 127) // 128, device=dev)
                sb = torch.empty((K + 127) // 128, (N + 127) // 128, device=dev)
                pgk.quant_fp8(Ad, a, sa, 0, stream=sh)
                pgk.quant_fp8(Bd, b, sb, 1, stream=sh)
                k = lambda: pgk.gemm_lowp(M, N, K, dt, a, Kp, b, Kp, C, N, scaleA=sa, scaleB=sb,
                                          prog=best, stream=sh)
            elif dt == pgk.BF16:
                a = torch.empty(M, Kp, dtype=torch.int16, device=dev)
                b = torch.empty(N, Kp, dtype=torch.int16, device=dev)
                pgk.cvt_bf16(Ad, a, 0, stream=sh)
                pgk.cvt_bf16(Bd, b, 1, stream=sh)
                k = lambda: pgk.gemm_lowp(M, N, K, dt, a, Kp, b, Kp, C, N, prog=best, stream=sh)
            else:
                a = torch.empty(M, Kp, dtype=torch.int16, device=dev)
                al = torch.empty_like(a)
                b = torch.empty(N, Kp, dtype=torch.int16, device=dev)
                bl = torch.empty_like(b)
                pgk.split_bf16(Ad, a, al, 0, stream=sh)
                pgk.split_bf16(Bd, b, bl, 1, stream=sh)
                k = lambda: pgk.gemm_lowp(M, N, K, dt, a, Kp, b, Kp, C, N, A_lo=al, Bt_lo=bl,
                                          prog=best, stream=sh)
            k()
            kern_ms = _events_ms(k, 10, stream)
        fl = 2.0 * M * N * K
        out.append({"shape": [M, N, K], "dist": dist, "form": name, "params": list(best.as_tuple()),
                    "step_ms": step_ms, "step_tflops": fl / step_ms / 1e9,
                    "step_gbs_fp32_io": 4.0 * (M * K + K * N + M * N) / step_ms / 1e6,
                    "kernel_ms": kern_ms, "kernel_pipe_tflops": pipe / 2 * fl / kern_ms / 1e9,
                    "rel_err_64_rows": err})
    del Ad, Bd, C
    torch.cuda.empty_cache()
    return out


def precision(dev, stream):
    import torch
    out = []
    for dist in ("normal", "normal_rowscaled"):
        out += _forms_at(8192, 8192, 8192, dist, dev, stream)
    return {"config": "precision 8192^3", "results": out}


def forms(dev, stream):
    """Every form at the other FP32 shapes (uniform[-1,1], seeds 0 / 1)."""
    out = []
    for M, N, K in ((4096, 4096, 4096), (8192, 1024, 4096), (16384, 64, 16384)):
        out += _forms_at(M, N, K, "uniform", dev, stream)
    return {"config": "forms at 4096^3, 8192x1024x4096, 16384x64x16384", "results": out}


def mm_table(dev, stream):
    """GB300 counterpart of the paper's Table "mm": the int32 paper-form kernel at
    n = 2^10 and 2^11 for the paper's (ub1, B0) x s grid (tile = B0), plus the
    tuned int32 register-blocked kernel; time and int32 Gop/s (2 n^3 / t)."""
    import torch
    grid = [(16, 4), (32, 4), (64, 4), (8, 8), (16, 8), (32, 8), (64, 8)]
    rng = np.random.default_rng(0)
    out = []
    sh = stream.cuda_stream
    if ONLY is not None:
        grid = [(ONLY[1], ONLY[0])]
    for n in ((2048,) if ONLY is not None else (1024, 2048)):
        A = torch.from_numpy(rng.integers(-100, 100, size=(n, n)).astype(np.int32)).to(dev)
        B = torch.from_numpy(rng.integers(-100, 100, size=(n, n)).astype(np.int32)).to(dev)
        C = torch.empty(n, n, dtype=torch.int32, device=dev)
        rows = []
        for ub1, b0 in grid:
            for s in ((ONLY[2],) if ONLY is not None else (2, 4)):
                p = pgk.params(*ONLY) if ONLY is not None else pgk.params(b0, ub1, s)
                run = lambda: pgk.gemm_i32(A, B, C, p, stream=sh)
                run()
                ms = _events_ms(run, 10, stream)
                rows.append({"ub1": ub1, "B0": b0, "s": s, "ms": ms, "gops": 2.0 * n ** 3 / ms / 1e6})
        best = min(rows, key=lambda r: r["ms"])
        if ONLY is not None:
            out.append({"n": n, "paper_grid": rows})
            continue
        cands = pgk.default_candidates(pgk.I32)
        tuned, _ = pgk.autotune(A, B, C, pgk.I32, candidates=[c for c in cands if c.sr > 1], reps=3,
                                stream=stream)
        run = lambda: pgk.gemm_i32(A, B, C, tuned, stream=sh)
        run()
        tms = _events_ms(run, 10, stream)
        out.append({"n": n, "paper_grid": rows, "best_paper_form": best,
                    "tuned_register_blocked": {"params": list(tuned.as_tuple()), "ms": tms,
                                               "gops": 2.0 * n ** 3 / tms / 1e6}})
    return {"config": "Table mm counterpart, int32", "sizes": out}


def transpose_table(dev, stream):
    """GB300 counterpart of the paper's transposition table: order 2^14 on 32-bit
    words, (B0, B1) in {(4,32), (8,32), (16,32), (32,32)} x granularity {2, 4, 8};
    time and GB/s of compulsory traffic (read a, write c: 2 x 4 n^2 bytes)."""
    import torch
    n = 16384
    a = torch.randint(-2 ** 31, 2 ** 31 - 1, (n, n), dtype=torch.int32, device=dev)
    c = torch.empty(n, n, dtype=torch.int32, device=dev)
    sh = stream.cuda_stream
    rows = []
    for b0, b1 in ([tuple(ONLY[:2])] if ONLY is not None else ((4, 32), (8, 32), (16, 32), (32, 32))):
        for s in ((ONLY[2],) if ONLY is not None else (2, 4, 8)):
            p = pgk.params(b0, b1, s)
            run = lambda: pgk.transpose(a, c, p, stream=sh)
            run()
            ms = _events_ms(run, 10, stream)
            rows.append({"B0": b0, "B1": b1, "s": s, "ms": ms, "gbs": 8.0 * n * n / ms / 1e6})
    best = min(rows, key=lambda r: r["ms"])
    return {"config": "transposition order 2^14", "grid": rows, "best": best}


def jacobi_table(dev, stream):
    """GB300 counterpart of the paper's 1D Jacobi table: T = 4 steps on a vector of
    length 2^15 + 2, blocks 16-256 x granularity {2, 4, 8}; and the same grid on
    2^27 + 2 points, where the step is HBM-bound (4 + 4 bytes per point)."""
    import torch
    out = {}
    sh = stream.cuda_stream
    for n, steps in (((2 ** 27 + 2, 4),) if ONLY is not None else ((2 ** 15 + 2, 4), (2 ** 27 + 2, 4))):
        a = torch.randint(-2 ** 20, 2 ** 20, (2 * n,), dtype=torch.int32, device=dev)
        rows = []
        for b in ((ONLY[0],) if ONLY is not None else (16, 32, 64, 128, 256)):
            for s in ((ONLY[2],) if ONLY is not None else (2, 4, 8)):
                p = pgk.params(b, 1, s)
                run = lambda: pgk.jacobi(a, n, steps, p, stream=sh)
                run()
                ms = _events_ms(run, 10, stream)
                rows.append({"B": b, "s": s, "ms": ms, "ms_per_step": ms / steps,
                             "gbs": 8.0 * (n - 2) * steps / ms / 1e6})
        out[str(n)] = {"grid": rows, "best": min(rows, key=lambda r: r["ms"])}
    return {"config": "1D Jacobi", "sizes": out}


def errmeas(dev, stream):
    """FP64 relative-error reduction over an 8192 x 8192 FP32 result against an FP64
    reference: time and GB/s of its compulsory traffic (4 + 8 bytes per entry)."""
    import torch
    n = 8192
    C = torch.randn(n, n, device=dev)
    R = C.double() + 1e-3
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    run = lambda: pgk.relerr(C, R, out, stream=stream.cuda_stream)
    run()
    ms = _events_ms(run, 20, stream)
    return {"config": "relerr 8192^2", "ms": ms, "gbs": 12.0 * n * n / ms / 1e6}


def mlp_kernels(dev, stream):
    """Cost-model kernels: forward over 30 000 candidate rows, one minibatch
    gradient (256 rows) + Adam step, and a 15 000-row full-batch gradient."""
    import torch
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.standard_normal((30000, 7)).astype(np.float32)).to(dev)
    t = torch.from_numpy(rng.standard_normal(30000).astype(np.float32)).to(dev)
    th = torch.from_numpy(inputs.he_uniform_mlp(0)).to(dev)
    y = torch.empty(30000, device=dev)
    g = torch.zeros_like(th)
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    loss = torch.zeros(1, device=dev)
    sh = stream.cuda_stream
    idx = torch.arange(256, dtype=torch.int32, device=dev)
    fwd = lambda: pgk.mlp_forward(X, th, y, stream=sh)
    step = lambda: (pgk.mlp_loss_grad(X, t, th, g, loss, idx=idx, stream=sh),
                    pgk.mlp_adam(th, g, m, v, 1, stream=sh))
    full = lambda: pgk.mlp_loss_grad(X[:15000], t[:15000], th, g, loss, stream=sh)
    for f in (fwd, step, full):
        f()
    return {"config": "cost-model kernels", "forward_30000_ms": _events_ms(fwd, 20, stream),
            "minibatch_step_ms": _events_ms(step, 20, stream),
            "full_gradient_15000_ms": _events_ms(full, 20, stream)}


def _clock_sampler():
    import subprocess
    try:
        return subprocess.Popen(["nvidia-smi", "--query-gpu=clocks.sm", "--format=csv,noheader,nounits",
                                 "-i", "0", "-lms", "100"], stdout=subprocess.PIPE,
                                stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def _clock_median(proc):
    if proc is None:
        return None
    proc.terminate()
    out, _ = proc.communicate(timeout=10)
    vals = [float(x) for x in out.split() if x.strip().replace(".", "", 1).isdigit()]
    return statistics.median(vals) if vals else None


def peaks(dev, stream):
    """Measured denominators beside the derived ones.  The FP32 probe is the
    library's own kernel; the BF16 and FP8 matmuls are PyTorch's (cuBLAS), timed
    here only as context for the tensor-core fractions."""
    import torch
    m = pgk.machine_query(0)
    blocks = m.sm_count * 8
    sink = torch.empty(blocks * 256, device=dev)
    sh = stream.cuda_stream
    out = {"config": "peaks", "sm_count": m.sm_count}
    for paired in (1, 0):
        iters = 20000
        run = lambda: pgk.simt_peak_probe(blocks, iters, paired, sink, stream=sh)
        run()
        clk = _clock_sampler()
        ms = _events_ms(run, 12, stream)
        mhz = _clock_median(clk)
        flops = blocks * 256 * iters * 16 * (2 if paired else 1) * 2
        r = {"ms": ms, "tflops": flops / ms / 1e9, "sm_mhz": mhz}
        if mhz:
            r["tflops_per_ghz"] = r["tflops"] / (mhz / 1e3)
            r["derived_at_clock"] = m.sm_count * 128 * 2 * mhz * 1e6 / 1e12
        out["fma_probe_paired" if paired else "fma_probe_scalar"] = r
    n = 8192
    flops = 2.0 * n * n * n
    try:
        # FP32 SGEMM with TF32 off: context for the SIMT fraction
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        a = torch.randn(n, n, device=dev)
        b = torch.randn(n, n, device=dev)
        run = lambda: torch.matmul(a, b)
        for _ in range(3):
            run()
        clk = _clock_sampler()
        ms = _events_ms(run, 8, stream)
        out["torch_fp32_matmul"] = {"ms": ms, "tflops": flops / ms / 1e9, "sm_mhz": _clock_median(clk)}
        torch.backends.cuda.matmul.allow_tf32 = prev
        del a, b
    except Exception as e:  # context only
        out["torch_fp32_matmul"] = {"error": str(e)[:200]}
    try:
        a = torch.randn(n, n, device=dev, dtype=torch.bfloat16)
        b = torch.randn(n, n, device=dev, dtype=torch.bfloat16)
        run = lambda: torch.matmul(a, b)
        for _ in range(3):
            run()
        clk = _clock_sampler()
        ms = _events_ms(run, 20, stream)
        out["torch_bf16_matmul"] = {"ms": ms, "tflops": flops / ms / 1e9, "sm_mhz": _clock_median(clk)}
    except Exception as e:  # context only
        out["torch_bf16_matmul"] = {"error": str(e)[:200]}
    try:
        a8 = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn)
        b8 = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn).t()
        one = torch.ones((), device=dev)
        run = lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        for _ in range(3):
            run()
        clk = _clock_sampler()
        ms = _events_ms(run, 20, stream)
        out["torch_fp8_scaled_mm"] = {"ms": ms, "tflops": flops / ms / 1e9, "sm_mhz": _clock_median(clk)}
    except Exception as e:  # context only
        out["torch_fp8_scaled_mm"] = {"error": str(e)[:200]}
    return out


def link(dev, stream):
    """Host-link bandwidth with pinned buffers (PyTorch copies, timed with events on
    the copy streams) and the end-to-end step time of pgk_gemm_host at 8192^3."""
    import torch
    n = 64 * 1024 * 1024                       # 256 MiB of float32
    h_in = torch.empty(n).pin_memory()
    h_out = torch.empty(n).pin_memory()
    d_in = torch.empty(n, device=dev)
    d_out = torch.empty(n, device=dev)
    s2 = torch.cuda.Stream(device=dev)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            best = min(best, (time.perf_counter() - t0) * 1e3)
        return best

    def h2d():
        with torch.cuda.stream(stream):
            d_in.copy_(h_in, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s2):
            h_out.copy_(d_out, non_blocking=True)

    gb = n * 4 / 1e9
    out = {"config": "host link, pinned 256 MiB copies"}
    out["h2d_gbs"] = gb / timed(h2d) * 1e3
    out["d2h_gbs"] = gb / timed(d2h) * 1e3
    out["duplex_gbs_total"] = 2 * gb / timed(lambda: (h2d(), d2h())) * 1e3
    del h_in, h_out, d_in, d_out
    M = N = K = 8192
    A, B = inputs.gemm_operands(M, N, K, seed=0)
    Ah, Bh = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
    Ch = torch.empty(M, N).pin_memory()
    prog = pgk.params(128, 256, 4, 0, 0)
    call = lambda: pgk.gemm_host(Ah, Bh, Ch, pgk.SPLIT_BF16, prog, stream=stream.cuda_stream)
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    steps = 20
    t0 = time.perf_counter()
    for _ in range(steps):
        call()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    link_ms = (M * K + K * N + M * N) * 4 / 1e9 / out["duplex_gbs_total"] * 1e3
    out.update({"gemm_host_split_ms_per_step": ms, "gemm_host_split_tflops": 2.0 * M * N * K / ms / 1e9,
                "link_time_for_768MiB_at_duplex_ms": link_ms})
    return out


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("which", nargs="*", default=["config1", "scale", "grouped", "precision"])
    ap.add_argument("--only", default=None,
                    help="B0,B1,s[,sr,tile]: one program point of mm / transpose / jacobi (profiling)")
    args = ap.parse_args()
    global ONLY
    if args.only:
        ONLY = [int(x) for x in args.only.split(",")]
    os.makedirs(args.out, exist_ok=True)
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    fns = {"config1": config1, "scale": scale, "grouped": grouped, "precision": precision,
           "mm": mm_table, "transpose": transpose_table, "jacobi": jacobi_table,
           "errmeas": errmeas, "mlp": mlp_kernels, "peaks": peaks, "forms": forms, "link": link}
    for w in args.which:
        t0 = time.time()
        with torch.cuda.stream(stream):
            r = fns[w](dev, stream)
        r["wall_s"] = time.time() - t0
        with open(os.path.join(args.out, f"{w}.json"), "w") as f:
            json.dump(r, f)
        print(w, json.dumps(r)[:1500], flush=True)


if __name__ == "__main__":
    main()
