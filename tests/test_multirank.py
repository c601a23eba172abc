"""The multi-process (torchrun) path of bench.py, on CPU with the gloo backend: every
rank advances its own copy of the workload (weak scaling); the job's time is the max
over ranks and its work the updates of all ranks."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (r + 1) seconds for 10 steps of 100 updates each
    value, t_ms = bench.job_throughput(100, 10, 1000.0 * (rank + 1), world, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, value, t_ms))


def test_job_throughput_is_max_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, t_ms in out:
        assert t_ms == 2000.0                      # the slower rank's time on every rank
        assert value == 100 * 10 * 2 / 2.0         # both ranks' updates over that time


def test_job_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench
    value, t_ms = bench.job_throughput(100, 10, 500.0, 1)
    assert t_ms == 500.0 and value == 2000.0
