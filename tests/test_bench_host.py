"""Host-side logic of bench.py on CPU: the whole-job throughput of N ranks is
the sum of their units over the slowest rank's time (2 gloo ranks)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, t = bench.job_throughput(1.0 + rank, 100.0 * (rank + 1))
    q.put((rank, value, t))
    dist.destroy_process_group()


def test_job_throughput_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for _, value, t in res:
        assert t == 2.0                     # slowest rank
        assert value == pytest.approx(300.0 / 2.0)


def test_job_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(2.0, 10.0) == (5.0, 2.0)
