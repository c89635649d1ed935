"""The multi-process path of bench.py (independent replicas, one rank per
GPU) on CPU: world size 2 over gloo, max-over-ranks timing and whole-job
throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank)
    val = bench.whole_job_tflops(3.0e12, world, ms)
    q.put((rank, ms, val))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_use_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, val in res:
        assert ms == 15.0                                  # max over ranks
        assert abs(val - 2 * 3.0e12 / 15e-3 / 1e12) < 1e-9   # both ranks' work over the slowest time


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_tflops(1.1e12, 1, 1000.0) == pytest.approx(1.1)
