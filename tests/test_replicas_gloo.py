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


def _split_rank(rank, world, port, q):
    # each rank takes its block of columns of the N-1 and scenario workloads, steps its own columns
    # of a small scenario run with the oracle, and counts only the units it ran
    import numpy as np
    import torch.distributed as dist
    import bench
    import netgen
    from oracle import emt as oemt
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        blocks = {}
        for cfg in (3, 4):
            w = bench.multi_workload(cfg, world, rank)
            blocks[cfg] = (w["c0"], w["c1"], w["trips"], w["ss"], w["ls"])
        net = netgen.add_loads(netgen.small_network(24, 3), seed=5)
        R, T = 7, 6
        ss, ls = netgen.scenario_scales(net, R, seed=13)
        c0, c1 = bench.rank_columns(R, world, rank)
        nw = oemt.Network(net, bench.DT, want_tree=False)
        mine = {c: oemt.simulate(nw, T, [], solver="dense", src_scale=ss[c], load_scale=ls[c])[0]
                for c in range(c0, c1)}
        units = bench.job_units(net["n_bus"] * (c1 - c0) * T, world)
        reqs = bench.rank_share(list(range(23)), world, rank)
        parts = [None] * world
        dist.all_gather_object(parts, (blocks, mine, units, reqs))
        if rank == 0:
            q.put(parts)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_columns_split_over_ranks_cover_each_column_once(world):
    import numpy as np
    import bench
    import netgen
    from oracle import emt as oemt
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # workloads: the ranks' blocks, put together, are the one-rank workload
    for cfg in (3, 4):
        one = bench.multi_workload(cfg, 1, 0)
        got_trips, got_ss, got_ls, nxt = {}, [], [], 0
        for blocks, _, _, _ in parts:
            c0, c1, trips, ss, ls = blocks[cfg]
            assert c0 == nxt and c1 > c0
            nxt = c1
            got_trips.update({c0 + c: t for c, t in trips.items()})
            if ss is not None:
                got_ss.append(ss)
                got_ls.append(ls)
        assert nxt == one["R"]
        assert got_trips == one["trips"]
        if one["ss"] is not None:
            assert np.array_equal(np.concatenate(got_ss), one["ss"])
            assert np.array_equal(np.concatenate(got_ls), one["ls"])
    # a run: the union of the ranks' columns equals the one-rank run, and the job's units count
    # every column once
    net = netgen.add_loads(netgen.small_network(24, 3), seed=5)
    R, T = 7, 6
    ss, ls = netgen.scenario_scales(net, R, seed=13)
    nw = oemt.Network(net, bench.DT, want_tree=False)
    union = {}
    for _, mine, units, _ in parts:
        assert not (set(mine) & set(union))
        union.update(mine)
        assert units == net["n_bus"] * R * T
    assert sorted(union) == list(range(R))
    for c in range(R):
        ref, _ = oemt.simulate(nw, T, [], solver="dense", src_scale=ss[c], load_scale=ls[c])
        assert np.array_equal(union[c], ref)
    # the request stream: every request served by exactly one rank
    served = sorted(i for _, _, _, reqs in parts for i, _ in reqs)
    assert served == list(range(23))


def test_accuracy_columns_span_the_tile_edges():
    import bench
    assert bench.accuracy_columns(512) == [0, 1, 191, 192, 256, 447, 510, 511]
    assert bench.accuracy_columns(64) == [0, 1, 32, 62, 63]
    assert bench.rank_columns(512, 3, 0) == (0, 170) and bench.rank_columns(512, 3, 2) == (341, 512)
