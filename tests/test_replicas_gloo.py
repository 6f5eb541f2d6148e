"""The N > 1 host path of bench.py on CPU: two gloo ranks, each reporting its
own time and cells; the job throughput is all cells over the slowest time."""
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


def _rank(rank, world, port, q):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_0910_2854_gb300.replicas import job_throughput
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rate, ms = job_throughput(10.0 + rank, 100 * (rank + 1))
    q.put((rank, rate, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, rate, ms in res:
        assert ms == 11.0
        assert rate == pytest.approx(300 / 11e-3)


def test_single_process_returns_its_own():
    from paper_0910_2854_gb300.replicas import job_throughput
    rate, ms = job_throughput(5.0, 1000)
    assert ms == 5.0 and rate == pytest.approx(1000 / 5e-3)
