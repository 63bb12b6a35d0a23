"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the timed
value is the slowest rank's, the job throughput counts every rank's
replica, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
        worst = bench.max_over_ranks(ms, dist, "cpu")
        value = bench.job_throughput(4.0e6, world, worst)

        class A:
            steps, warmup, cpu_rows = 1, 0, 3
        rc = bench.run_reference(A, world, rank) if rank != 0 else None
        q.put((rank, worst, value, rc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, worst, value, rc in res:
        assert worst == 15.0                          # max over ranks, seen by every rank
        assert abs(value - 2 * 4.0e6 / 15e-3 / 1e6) < 1e-9
        if rank != 0:
            assert rc == 0                            # non-zero ranks skip the reference arm
