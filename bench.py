"""Benchmark of the parametric GEMM hot path on GB300.

One step = one GEMM C = A*B at M = N = K = 8192 (FP32 inputs, FP32 output) in
the chosen arithmetic form (default: split BF16, three BF16 products with FP32
accumulation, FP32-level accuracy), with every stage of the path inside the
step: operand preparation (for the tensor-core forms) and the GEMM kernel; the
case discussion runs on the host before each launch.  Inputs (256 MiB each)
exceed the 129 MB L2, so no flush is needed between steps.

The metric compares the chosen form with the plain FP32 parametric GEMM tuned
exhaustively over its register-blocked variants: both arms are autotuned and
timed on the same operands in the same run, and both report their relative
Frobenius error and largest per-row relative error on 64 rows against the FP64
oracle.  If the chosen form misses its tolerance the headline is the FP32 arm.

Prints ONE JSON line (rank 0).  `value` is whole-job TFLOP/s (2 M N K per GEMM,
all ranks), `roofline` describes the dominant kernel (the GEMM),
`config.fp32_tuned` the FP32 arm (with its own roofline against the SIMT peak),
`cpu_baseline` the FP64 CPU oracle on a bounded sample of rows of the same
product.  The oracle runs only in that leg (`oracle_leg`), which also yields the
reference rows of the error columns.

--impl reference times the oracle itself (the CPU reference arm) on the same
workload, a bounded sample of rows per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MEASURED_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                     "sm_max_mhz": 2070.0}
METRIC = "GEMM TFLOP/s & % roofline, chosen form vs plain FP32 tuned, at stated rel. error"
FORM_NAMES = {"f32": "FP32 SIMT (register-blocked parametric kernel)",
              "split": "split-BF16 (3 BF16 products, tcgen05, FP32 accumulate)",
              "bf16": "BF16 tcgen05, FP32 accumulate",
              "fp8": "FP8-E4M3 per-128x128-tile scaled tcgen05, FP32 accumulate"}
# the arithmetic each form computes in: split = three BF16 products (hi*hi, hi*lo,
# lo*hi) accumulated in FP32, FP32-level accuracy
FORM_DTYPE = {"f32": "f32", "split": "bf16x3-split (fp32 accumulate)",
              "bf16": "bf16 (fp32 accumulate)", "fp8": "fp8-e4m3 (fp32 accumulate)"}
FORM_TOL = {"f32": 1e-5, "split": 2e-5, "bf16": 2e-2, "fp8": 5e-2}


def peaks():
    p = dict(MEASURED_FALLBACK)
    src = "fallback"
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p.update(json.load(f))
        src = "measured"
    return p, src


class ClockSampler:
    """nvidia-smi sampling every 50 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_leg(A, B, err_rows, timed, target_s=12.0):
    """The CPU-oracle leg: the FP64 oracle's rows `err_rows` of A*B (the reference
    for the error columns) and, when `timed`, the oracle timed on a bounded sample
    of full output rows (the cpu_baseline)."""
    import numpy as np

    import oracle
    oracle.build()
    ref = oracle.gemm(A, B, rows=err_rows)
    if not timed:
        return ref, None
    M, K = A.shape
    N = B.shape[1]
    cores = oracle.max_threads()
    # calibrate with one row per core (the oracle parallelises over rows)
    rows = np.linspace(0, M - 1, cores).astype(np.int64)
    t0 = time.perf_counter()
    oracle.gemm(A, B, rows=rows)
    per_row = (time.perf_counter() - t0) / cores
    nrows = int(min(M, round(target_s / max(per_row, 1e-9))))
    nrows = max(cores, (nrows // cores) * cores)
    rows = np.linspace(0, M - 1, nrows).astype(np.int64)
    t0 = time.perf_counter()
    oracle.gemm(A, B, rows=rows)
    dt = time.perf_counter() - t0
    flops = 2.0 * nrows * N * K
    return ref, {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                 "sample": f"{nrows} of {M} output rows of the {M}x{N}x{K} product in FP64 "
                           f"(i-k-j loop, OpenMP), {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_1801_04348_gb300 import inputs
    M, N, K = gemm_shape(args)
    A, B = inputs.gemm_operands(M, N, K, seed=0)
    oracle.build()
    cores = oracle.max_threads()
    # bounded sample per step so that the whole run stays within a few minutes
    per_step_rows = max(cores, 2 * cores)
    rows_all = np.linspace(0, M - 1, per_step_rows * (args.steps + args.warmup)).astype(np.int64)
    for w in range(args.warmup):
        oracle.gemm(A, B, rows=rows_all[w * per_step_rows:(w + 1) * per_step_rows])
    times = []
    for s in range(args.steps):
        r = rows_all[(args.warmup + s) * per_step_rows:(args.warmup + s + 1) * per_step_rows]
        t0 = time.perf_counter()
        oracle.gemm(A, B, rows=r)
        times.append(time.perf_counter() - t0)
    flops = 2.0 * per_step_rows * N * K
    tot = sum(times)
    value = flops * len(times) / tot / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{M}x{N}x{K} FP32-input GEMM, FP64 CPU oracle, "
                                   f"{per_step_rows} sampled output rows per step",
                       "M": M, "N": N, "K": K},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step_rows} of {M} output rows per step"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def row_errors(got, ref):
    """(relative Frobenius error, largest per-row relative error) of sampled rows."""
    import numpy as np
    got = np.asarray(got, dtype=np.float64)
    d = np.linalg.norm(got - ref, axis=1)
    r = np.linalg.norm(ref, axis=1)
    frob = float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))
    return frob, float(np.max(d / np.maximum(r, 1e-300)))


def time_arm(step, gemm_events, steps, warmup, stream, dev, ws, local):
    """W untimed steps, ~0.6 s of untimed steps while the clock sampler starts, then
    `steps` steps between a barrier and a synchronise, timed with CUDA events on
    the launching stream.  Returns (ms, per-GEMM ms list, clocks)."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    torch.cuda.synchronize(dev)
    # nvidia-smi needs a moment to start: keep the GPU busy with extra untimed
    # steps for ~0.6 s after starting it, so the samples see the kernel under load
    sampler = ClockSampler(local)
    sampler.start()
    t_busy = time.perf_counter()
    with torch.cuda.stream(stream):
        while time.perf_counter() - t_busy < 0.6:
            step()
            torch.cuda.synchronize(dev)
    gemm_events.clear()
    if ws > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    gemm_ms = [a.elapsed_time(b) for a, b in gemm_events[-steps:]] if gemm_events else []
    return ms, gemm_ms, clocks


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0,
                    help="timed steps (0 = as many as fill about 3 s)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="split", choices=["split", "f32", "bf16", "fp8"],
                    help="the chosen arithmetic form (the headline); the tuned FP32 arm is "
                         "measured beside it")
    ap.add_argument("--size", type=int, default=8192)
    ap.add_argument("--shape", default=None,
                    help="M,N,K of the GEMM (default: --size for all three); other shapes than "
                         "8192^3 are measurements beside the benchmark workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32-arm", action="store_true",
                    help="skip the tuned FP32 arm (the comparison the metric names)")
    ap.add_argument("--tune-log", default=None, help="append the autotuner's CSV rows here")
    ap.add_argument("--params", default=None,
                    help="B0,B1,s,sr,tile: use these program parameters instead of autotuning")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    from paper_1801_04348_gb300 import build as pbuild
    from paper_1801_04348_gb300 import inputs, pgk

    ws, rank, local = dist_env()
    pbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    M, N, K = gemm_shape(args)
    A, B = inputs.gemm_operands(M, N, K, seed=rank)
    Ad = torch.from_numpy(A).to(dev)
    Bd = torch.from_numpy(B).to(dev)
    C = torch.empty(M, N, device=dev)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    machine = pgk.machine_query(local)
    err_rows = np.linspace(0, M - 1, 64).astype(np.int64)
    err_rows_d = torch.from_numpy(err_rows).to(dev)

    form = args.form
    fixed = pgk.params(*[int(x) for x in args.params.split(",")]) if args.params else None
    if fixed is None and form in ("split", "bf16") and N <= 64:
        # skinny products: the library's case discussion takes the fused-conversion
        # program and its K slices (prog = None), which no fixed candidate list holds
        prog = None
    else:
        prog = tune_form(form, Ad, Bd, C, stream, pgk, torch, fixed, args.tune_log)
    step, gemm_events, launches_per_step, alg = make_step(form, prog, Ad, Bd, C, M, N, K, sh, pgk,
                                                          torch, dev)
    if args.steps <= 0:
        with torch.cuda.stream(stream):
            step()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            step()
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t0
        args.steps = int(min(2000, max(10, 3.0 / max(dt, 1e-6))))
    ms, gemm_ms, clocks = time_arm(step, gemm_events, args.steps, args.warmup, stream, dev, ws, local)
    got_form = C[err_rows_d].cpu().numpy()
    t_max = max_over_ranks(ms / 1e3, dev, ws)
    value = whole_job_tflops(2.0 * M * N * K * args.steps, t_max, ws)

    pk, pk_src = peaks()
    roof = roofline(form, alg, gemm_ms, ms / args.steps, machine, pk, pk_src, clocks,
                    recorded_traffic(form, prog, (M, N, K)) if prog is not None else None,
                    timed_s=ms / 1e3)

    # the comparison the metric names: plain FP32 SIMT, exhaustively tuned over the
    # register-blocked family, on the same operands
    arm32 = None
    if form != "f32" and not args.no_fp32_arm:
        C32 = torch.empty(M, N, device=dev)
        prog32 = tune_form("f32", Ad, Bd, C32, stream, pgk, torch, None, args.tune_log)
        step32, ev32, l32, alg32 = make_step("f32", prog32, Ad, Bd, C32, M, N, K, sh, pgk, torch,
                                             dev)
        steps32 = max(10, min(args.steps, 40))
        ms32, gms32, clocks32 = time_arm(step32, ev32, steps32, args.warmup, stream, dev, ws, local)
        t32 = max_over_ranks(ms32 / 1e3, dev, ws)
        roof32 = roofline("f32", alg32, gms32, ms32 / steps32, machine, pk, pk_src, clocks32,
                          recorded_traffic("f32", prog32, (M, N, K)), timed_s=ms32 / 1e3)
        arm32 = {"value": whole_job_tflops(2.0 * M * N * K * steps32, t32, ws), "unit": "TFLOP/s",
                 "ms_per_step": t32 * 1e3 / steps32, "steps": steps32,
                 "program_params": list(prog32.as_tuple()), "roofline": roof32,
                 "gpu_launches": l32 * steps32, "clocks": clocks32,
                 "got": C32[err_rows_d].cpu().numpy()}
        del C32

    # end to end: host (pinned) inputs -> device -> GEMM -> host result
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(form, prog, A, B, M, N, K, dev, stream, pgk, torch, args, ws)

    cpu = None
    errs = None
    if rank == 0:
        ref, cpu = oracle_leg(A, B, err_rows, timed=(ws == 1 and not args.no_cpu_baseline))
        errs = {"form": row_errors(got_form, ref)}
        if arm32 is not None:
            errs["f32"] = row_errors(arm32.pop("got"), ref)
    elif arm32 is not None:
        arm32.pop("got")
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank != 0:
        return 0
    err, err_row = errs["form"]
    met = err <= FORM_TOL[form]
    config = {"workload": f"{M}x{N}x{K} GEMM, FP32 in/out, uniform[-1,1] seed 0(+rank), "
                          f"form: {FORM_NAMES[form]}",
              "M": M, "N": N, "K": K, "form": form,
              "program_params": (list(prog.as_tuple()) if prog is not None else
                                 "case discussion: fused-conversion program, K slices to fill the SMs"),
              "rel_frobenius_err": err, "max_row_rel_err": err_row,
              "err_sample": f"{len(err_rows)} rows against the FP64 oracle",
              "tolerance": FORM_TOL[form], "tolerance_met": met,
              "l2": "inputs 256 MiB each > 129 MB L2; no flush"}
    line = {
        "metric": METRIC,
        "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": FORM_DTYPE[form], "data": "synthetic",
        "config": config, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
    }
    if arm32 is not None:
        e32, r32 = errs["f32"]
        arm32.update({"rel_frobenius_err": e32, "max_row_rel_err": r32, "tolerance": FORM_TOL["f32"],
                      "tolerance_met": e32 <= FORM_TOL["f32"]})
        config["fp32_tuned"] = arm32
        line["speedup_vs_fp32_tuned"] = value / arm32["value"]
    if not met:
        # the chosen form missed its accuracy: the headline is the tuned FP32 arm
        line["chosen_form_missed_tolerance"] = True
        if arm32 is not None:
            line["value"] = arm32["value"]
            line["ms_per_step"] = arm32["ms_per_step"]
            line["dtype"] = FORM_DTYPE["f32"]
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(t_local, device, ws):
    """Slowest rank's time (seconds): every rank ran the same number of steps
    between the same barriers, so the job takes as long as its slowest rank."""
    if ws <= 1:
        return t_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_local], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(flops_per_rank, t_max, ws):
    """Weak scaling: each rank does its own GEMMs; whole-job rate = all ranks'
    flops over the slowest rank's time."""
    return flops_per_rank * ws / t_max / 1e12


def tune_form(form, Ad, Bd, C, stream, pgk, torch, fixed=None, tune_log=None):
    """Program parameters of the form for this shape: `fixed`, else the autotuner's
    fastest candidate on the real operands (FP32: the register-blocked family)."""
    dt = {"f32": pgk.F32, "split": pgk.SPLIT_BF16, "bf16": pgk.BF16, "fp8": pgk.FP8_E4M3}[form]
    if fixed is not None:
        return fixed
    if form == "f32":
        cands = [p for p in pgk.default_candidates(dt) if p.sr > 1]
    else:
        cands = pgk.default_candidates(dt)
    with torch.cuda.stream(stream):
        best, _ = pgk.autotune(Ad, Bd, C, dt, candidates=cands, reps=2, stream=stream,
                               log_path=tune_log)
    torch.cuda.synchronize()
    return best


def make_step(form, prog, Ad, Bd, C, M, N, K, sh, pgk, torch, dev):
    """Returns (step callable, list of (start, end) events around the GEMM
    kernel, kernel launches per step, algorithmic work per GEMM launch)."""
    events = []
    if form == "f32":
        def step():
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            pgk.gemm(Ad, Bd, C, pgk.F32, prog, stream=sh)
            b.record()
            events.append((a, b))
        return step, events, 1, {"flops": 2.0 * M * N * K}
    if (prog is None or prog.B1 == 64) and form in ("split", "bf16"):
        # the fused-conversion program: one library call converts B^T and runs the
        # GEMM, which reads A in FP32 itself (HBM-bound: A crosses memory once)
        dt = pgk.SPLIT_BF16 if form == "split" else pgk.BF16

        def step():
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            pgk.gemm(Ad, Bd, C, dt, prog, stream=sh)
            b.record()
            events.append((a, b))
        return step, events, 2, {"flops": (6.0 if form == "split" else 2.0) * M * N * K,
                                 "bytes": 4.0 * (M * K + K * N + M * N)}
    Kp = (K + 15) // 16 * 16
    if form == "split":
        Ah = torch.empty(M, Kp, dtype=torch.int16, device=dev)
        Al = torch.empty_like(Ah)
        Bh = torch.empty(N, Kp, dtype=torch.int16, device=dev)
        Bl = torch.empty_like(Bh)

        def step():
            pgk.split_bf16(Ad, Ah, Al, 0, stream=sh)
            pgk.split_bf16(Bd, Bh, Bl, 1, stream=sh)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            pgk.gemm_lowp(M, N, K, pgk.SPLIT_BF16, Ah, Kp, Bh, Kp, C, N, A_lo=Al, Bt_lo=Bl,
                          prog=prog, stream=sh)
            b.record()
            events.append((a, b))
        return step, events, 3, {"flops": 6.0 * M * N * K}
    if form == "bf16":
        Ah = torch.empty(M, Kp, dtype=torch.int16, device=dev)
        Bh = torch.empty(N, Kp, dtype=torch.int16, device=dev)

        def step():
            pgk.cvt_bf16(Ad, Ah, 0, stream=sh)
            pgk.cvt_bf16(Bd, Bh, 1, stream=sh)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            pgk.gemm_lowp(M, N, K, pgk.BF16, Ah, Kp, Bh, Kp, C, N, prog=prog, stream=sh)
            b.record()
            events.append((a, b))
        return step, events, 3, {"flops": 2.0 * M * N * K}
    Aq = torch.empty(M, Kp, dtype=torch.uint8, device=dev)
    Bq = torch.empty(N, Kp, dtype=torch.uint8, device=dev)
    sA = torch.empty((M + 127) // 128, (K + 127) // 128, device=dev)
    sB = torch.empty((K + 127) // 128, (N + 127) // 128, device=dev)

    def step():
        pgk.quant_fp8(Ad, Aq, sA, 0, stream=sh)
        pgk.quant_fp8(Bd, Bq, sB, 1, stream=sh)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        pgk.gemm_lowp(M, N, K, pgk.FP8_E4M3, Aq, Kp, Bq, Kp, C, N, scaleA=sA, scaleB=sB, prog=prog,
                      stream=sh)
        b.record()
        events.append((a, b))
    return step, events, 3, {"flops": 2.0 * M * N * K}


KERNEL_SOURCES = {"f32": ["simt_rb.cuh", "simt_f32.cu"], "split": ["tc_gemm.cu"],
                  "bf16": ["tc_gemm.cu"], "fp8": ["tc_gemm.cu"]}


def gemm_shape(args):
    if args.shape:
        M, N, K = (int(x) for x in args.shape.split(","))
        return M, N, K
    return args.size, args.size, args.size


def recorded_traffic(form, prog, shape):
    """DRAM bytes per GEMM launch from the committed ncu summary
    profiles/traffic_<form>_<B0>-<B1>-<s>-<sr>-<tile>.txt, or None when that
    summary is missing, was taken on another shape, or the kernel source changed
    since it was taken."""
    import hashlib
    tag = "-".join(str(x) for x in prog.as_tuple())
    path = os.path.join(ROOT, "profiles", f"traffic_{form}_{tag}.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as f:
        for line in f:
            parts = line.split(None, 1)
            if len(parts) == 2:
                rec[parts[0]] = parts[1].strip()
    h = hashlib.sha1()
    for src in KERNEL_SOURCES[form]:
        with open(os.path.join(ROOT, "paper_1801_04348_gb300", "csrc", src), "rb") as f:
            h.update(f.read())
    if rec.get("source_sha1") != h.hexdigest():
        return None
    if rec.get("program_params") != ",".join(str(x) for x in prog.as_tuple()):
        return None
    if rec.get("shape") != ",".join(str(x) for x in shape):
        return None
    try:
        return float(rec["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def roofline(form, alg, gemm_ms, step_ms, machine, pk, pk_src, clocks, traffic=None, timed_s=0.0):
    kern_ms = statistics.mean(gemm_ms) if gemm_ms else step_ms
    if "bytes" in alg:
        # fused-conversion program: bound by reading A (FP32) once from HBM
        achieved = alg["bytes"] / (kern_ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                "kernel": "k_tc_gemm fused conversion (B^T conversion + GEMM, one call)",
                "peak_source": f"hbm copy ({pk_src})", "bytes_per_launch": alg["bytes"],
                "pipe_tflops": alg["flops"] / (kern_ms * 1e-3) / 1e12}
    achieved = alg["flops"] / (kern_ms * 1e-3) / 1e12
    if form == "f32":
        f = pk.get("sm_max_mhz", 2070.0)
        peak = machine.sm_count * 128 * 2 * f * 1e6 / 1e12
        out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
               "frac": achieved / peak, "traffic": traffic,
               "kernel": "k_rb (register-blocked FP32 SIMT)",
               "peak_source": f"{machine.sm_count} SMs x 128 FP32 lanes x 2 flop x {f:.0f} MHz "
                              f"(max SM clock, {pk_src})"}
        if clocks.get("sm_mhz"):
            out["frac_at_observed_clock"] = achieved / (peak * clocks["sm_mhz"] / f)
        return out
    # a kernel timed inside a long run (here >= 1 s of back-to-back steps) is held
    # to the sustained peak; a short burst to the burst peak
    sustained = timed_s >= 1.0
    base = pk["bf16_tflops_sustained"] if sustained else pk["bf16_tflops"]
    kind = "sustained" if sustained else "burst"
    mult = 2.0 if form == "fp8" else 1.0
    peak = mult * base
    src = (f"{'2 x ' if form == 'fp8' else ''}bf16 {kind} ({pk_src}, timed region {timed_s:.3f} s)"
           + ("; FP8 dense = 2x BF16 nominal" if form == "fp8" else ""))
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": "k_tc_gemm (tcgen05)",
            "peak_source": src, "flops_per_launch": alg["flops"],
            "frac_of_burst": achieved / (mult * pk["bf16_tflops"]),
            "frac_of_sustained": achieved / (mult * pk["bf16_tflops_sustained"])}


def measure_e2e(form, prog, A, B, M, N, K, dev, stream, pgk, torch, args, ws):
    """Same metric through the library's host-buffer call pgk_gemm_host: every
    step passes pinned host A and B and a pinned host C; the library copies the
    inputs to the device on its own stream (overlapping the previous step's GEMM)
    and the GEMM writes C back into host memory.  Timed on the host clock from
    the first call to the completion of the last, with the device idle before."""
    import time
    Ah = torch.from_numpy(A).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    Ch = torch.empty(M, N, dtype=torch.float32).pin_memory()
    dt = {"f32": pgk.F32, "split": pgk.SPLIT_BF16, "bf16": pgk.BF16, "fp8": pgk.FP8_E4M3}[form]
    steps = max(6, min(args.steps, 40))
    sh = stream.cuda_stream
    for _ in range(3):
        pgk.gemm_host(Ah, Bh, Ch, dt, prog, stream=sh)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        pgk.gemm_host(Ah, Bh, Ch, dt, prog, stream=sh)
    torch.cuda.synchronize(dev)
    ms = (time.perf_counter() - t0) * 1e3 / steps
    return {"value": 2.0 * M * N * K * ws / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
            "h2d_bytes_per_step": (M * K + K * N) * 4, "d2h_bytes_per_step": M * N * 4,
            "steps": steps, "ms_per_step": ms, "api": "pgk_gemm_host (pinned host A, B, C)",
            "pipelining": "input copies of step i+1 on the library's stream overlap the GEMM of step i; "
                          "the GEMM runs in row panels of whole tile rounds and each panel's C is "
                          "copied back while the next panel computes",
            "timing": "host clock, device idle before the first call, synchronised after the last"}


if __name__ == "__main__":
    sys.exit(main())
