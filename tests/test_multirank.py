"""Host logic of a multi-GPU benchmark run (replicas: each rank steps the whole workload on its own GPU, no
collective on the data path): the job's time is the slowest rank's and the throughput counts every rank's
cells.  Two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        own = [12.5, 20.0][rank]
        t = bench.job_time_ms(own, world, device="cpu")
        out.put((rank, t, bench.job_glups(3 * 1024 * 1024, 100, world, t)))
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_throughput_counts_every_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]
    expected = 3 * 1024 * 1024 * 100 * 2 / (20.0e-3) / 1e9
    assert all(abs(r[2] - expected) < 1e-9 * expected for r in res)


def test_one_rank_keeps_its_own_time():
    import bench
    assert bench.job_time_ms(7.25, 1) == 7.25
    assert abs(bench.job_glups(1000, 10, 1, 1.0) - 1e-2) < 1e-15
