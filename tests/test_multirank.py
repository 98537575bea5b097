"""Host logic of the multi-rank benchmark on CPU ranks (gloo, world size 2):
replicas of the solve run independently, the job time is the slowest rank's and
the throughput counts the units of every rank."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    elapsed = [100.0, 250.0][rank]
    units = [1000, 3000][rank]
    value, tmax = bench.whole_job_value(elapsed, units)
    out.put((rank, value, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_value_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
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
    for _, value, tmax in res:
        assert tmax == 250.0
        assert abs(value - 4000 / 0.25) < 1e-9


def test_whole_job_value_single_process():
    import bench

    value, tmax = bench.whole_job_value(200.0, 500)
    assert tmax == 200.0 and abs(value - 2500.0) < 1e-12
