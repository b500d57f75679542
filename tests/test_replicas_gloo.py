"""Multi-process aggregation of the benchmark on CPU (gloo, world size 2).

The GPU path shards as independent replicas: each rank steps its own copy of
the network and no data-path collective exists. The only exchange is the
whole-job time, the maximum over ranks of each rank's timed region, from which
the whole-job rate (units of all ranks per second) follows.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        own = [3.0, 5.0, 4.0][rank]
        ms = bench.job_ms(own, world)
        q.put((rank, ms, bench.job_rate(1000.0, world, ms)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_job_time_is_max_over_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = max([3.0, 5.0, 4.0][:world])
    for _, ms, rate in out:
        assert ms == want
        assert rate == pytest.approx(world * 1000.0 / (want / 1e3))


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_ms(2.5, 1) == 2.5
    assert bench.job_rate(10.0, 1, 2.0) == pytest.approx(5000.0)
