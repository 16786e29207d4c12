"""The benchmark's multi-replica bookkeeping on CPU with two gloo ranks: the slowest
rank's time and the whole-job rate (the GPU path has no data-path collective: replicas
only)."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    el = 100.0 + 50.0 * rank  # rank 1 is the slow one
    m = bench.max_over_ranks(el, world, device="cpu")
    q.put((rank, m, bench.job_rate(64 * 10, world, m)))
    dist.destroy_process_group()


def test_two_replica_max_and_rate():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in out:
        assert m == 150.0
        assert rate == pytest.approx(64 * 10 * 2 / 0.150)
