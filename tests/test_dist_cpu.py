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
