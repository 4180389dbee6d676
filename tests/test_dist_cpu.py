"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks, max-over-ranks
timing and the whole-job (weak scaling) aggregate."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, q):
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    t_local = 1.0 + rank                      # rank 1 is the slow one
    t_max = bench.max_over_ranks(t_local, torch.device("cpu"), ws)
    dist.barrier()
    q.put((rank, t_max, bench.whole_job_tflops(4e12, t_max, ws)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t_max, tf in out:
        assert t_max == 2.0
        assert tf == pytest.approx(4e12 * 2 / 2.0 / 1e12)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(0.25, None, 1) == 0.25
    assert bench.whole_job_tflops(1e12, 0.5, 1) == pytest.approx(2.0)


def test_recorded_traffic_matches_workload_and_program():
    """The roofline's DRAM traffic comes from a committed capture only for the
    workload and program it was taken on (and while the kernel source is unchanged)."""
    import bench
    from paper_1801_04348_gb300 import pgk
    prog = pgk.params(128, 256, 4, 0, 0)
    assert bench.recorded_traffic("split", prog, (4096, 4096, 4096)) is None
    assert bench.recorded_traffic("split", prog, (8192, 8192, 4096)) is None
    assert bench.recorded_traffic("split", pgk.params(128, 256, 5, 0, 0), (8192, 8192, 8192)) is None
    t = bench.recorded_traffic("split", prog, (8192, 8192, 8192))
    assert t is None or t > 8e8    # at least the compulsory bytes of one launch


def test_shape_option():
    import bench

    class A:
        shape, size = None, 4096
    assert bench.gemm_shape(A) == (4096, 4096, 4096)
    A.shape = "16384,64,16384"
    assert bench.gemm_shape(A) == (16384, 64, 16384)


def test_row_errors_frobenius_and_worst_row():
    import numpy as np

    import bench
    ref = np.array([[1.0, 0.0], [0.0, 2.0]])
    got = np.array([[1.0, 0.1], [0.0, 2.0]])
    frob, worst = bench.row_errors(got, ref)
    assert frob == pytest.approx(0.1 / np.sqrt(5.0))
    assert worst == pytest.approx(0.1)


def test_roofline_bounds_and_peaks():
    """FP32 against the derived SIMT peak (ALU), the tensor forms against the
    measured BF16 peak (burst for a short timed region, sustained for a long one;
    FP8 at twice it), the fused-conversion programs against the HBM copy rate."""
    import bench

    class Mach:
        sm_count = 152
    pk = {"hbm_gbs": 6800.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1700.0,
          "sm_max_mhz": 2000.0}
    clocks = {"sm_mhz": 1000.0}
    r = bench.roofline("f32", {"flops": 2e12}, [40.0], 40.0, Mach, pk, "t", clocks)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(152 * 128 * 2 * 2000e6 / 1e12)
    assert r["achieved"] == pytest.approx(50.0)
    assert r["frac_at_observed_clock"] == pytest.approx(2 * r["frac"])
    r = bench.roofline("split", {"flops": 6e12}, [3.0], 3.5, Mach, pk, "t", clocks, timed_s=0.1)
    assert r["bound"] == "tensor" and r["peak"] == 2000.0 and r["achieved"] == pytest.approx(2000.0)
    r = bench.roofline("split", {"flops": 6e12}, [3.0], 3.5, Mach, pk, "t", clocks, timed_s=2.0)
    assert r["peak"] == 1700.0
    r = bench.roofline("fp8", {"flops": 2e12}, [1.0], 1.2, Mach, pk, "t", clocks, timed_s=0.1)
    assert r["peak"] == 4000.0
    r = bench.roofline("split", {"flops": 1e11, "bytes": 6.8e9}, [2.0], 2.0, Mach, pk, "t", clocks)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["frac"] == pytest.approx(0.5)


def test_reference_arm_prints_one_line():
    """`bench.py --impl reference` runs the oracle on the host (no GPU needed) and
    prints the contract's JSON line with the reference keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--size", "64", "--steps", "2", "--warmup", "3"],
                         capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    for key in ("metric", "unit", "n_gpus", "ms_per_step", "higher_is_better", "cpu_baseline", "e2e"):
        assert key in line
    assert line["e2e"]["h2d_bytes_per_step"] == 0
