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
