"""Host logic of the N > 1 benchmark path (replicas), on CPU with gloo, world size 2.

Each rank times its own replica; the job's time is the slowest rank's and the
job's throughput is the units of all ranks divided by it.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [2.0, 3.5][rank]
    m = bench.max_over_ranks(elapsed, "cpu")
    rate = bench.whole_job_rate(world, 10, 1000, m)
    out.put((rank, m, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in res:
        assert m == 3.5
        assert rate == pytest.approx(2 * 10 * 1000 / 3.5)


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(1.25, "cpu") == 1.25
    assert bench.whole_job_rate(1, 4, 100, 2.0) == 200.0
