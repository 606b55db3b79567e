"""The replica (N>1) timing logic of bench.py on CPU: two gloo ranks with different
timings agree on the slowest one, and the whole-job rate counts every rank's steps."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = 100.0 + 37.5 * rank
    got = bench.max_over_ranks(mine)
    rate = bench.whole_job_rate(10, world, got)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, rate))


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_rate(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = 100.0 + 37.5 * (world - 1)
    for rank, got, rate in res:
        assert got == slowest
        assert abs(rate - world * 10 / (slowest / 1e3)) < 1e-9


def test_single_process_passthrough():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
