"""The N > 1 path of bench.py on CPU: two gloo ranks, each an independent
replica, aggregate with a max over ranks (no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    m = bench.reduce_max(ms, dist, "cpu")
    out[rank] = (m, bench.job_value(world, 1000, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_value():
    mp = torch.multiprocessing.get_context("spawn")
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        m, v = out[r]
        assert m == 15.0
        assert abs(v - 2 * 1000 / 0.015) < 1e-6


def test_single_process_helpers():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.job_value(1, 50, 2.0) == 25000.0
