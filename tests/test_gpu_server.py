"""Continuous-batching server: each request's result is the same alone and in a
mix (within the stated tolerance), and matches the CPU oracle."""
import numpy as np
import pytest

import netgen
from oracle import emt as oemt
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = 50e-6


@pytest.fixture(scope="module")
def L():
    from paper_2105_10661_gb300 import buildlib
    buildlib.build()
    import paper_2105_10661_gb300._lib as lib
    assert torch.cuda.is_available()
    return lib


NETS = {"a": (lambda: netgen.tile(1_000_000), 2), "b": (lambda: netgen.tiled(2, 2), 2)}


def _requests():
    # (network, arrival s, steps, kind, target, value, event step, length)
    ra = netgen.tile(1_000_000)
    rb = netgen.tiled(2, 2)
    ea = netgen.pick_branches(ra, 3, seed=3)
    eb = netgen.pick_branches(rb, 3, seed=4)
    return [
        ("a", 0.00, 180, 0, int(ea[0]), 0.0, 60, 0),
        ("a", 0.00, 120, 1, 17, 10.0, 20, 40),
        ("b", 0.00, 150, 0, int(eb[0]), 0.0, 100, 0),
        ("a", 0.02, 200, -1, 0, 0.0, 0, 0),
        ("b", 0.03, 130, 1, 101, 10.0, 30, 50),
        ("a", 0.05, 90, 0, int(ea[1]), 0.0, 45, 0),
        ("b", 0.06, 170, 0, int(eb[1]), 0.0, 10, 0),
        ("a", 0.08, 140, 1, 5, 10.0, 70, 30),
    ]


def _serve(L, reqs, tick=40):
    srv = L.emt_server_create(tick, 0)
    ids = {}
    mon = {}
    for key, (mk, levels) in NETS.items():
        net = mk()
        mon[key] = np.arange(0, net["n_bus"], 11)
        ids[key] = L.emt_server_add_network(srv, net, DT, levels=levels, max_slots=8, monitor=mon[key])
    rid = [L.emt_server_submit(srv, ids[r[0]], *r[1:]) for r in reqs]
    L.emt_server_run(srv)
    out = [L.emt_server_result(srv, i)[0] for i in rid]
    return out, L.emt_server_stats(srv), mon


def test_server_alone_equals_mixed_and_oracle(L):
    reqs = _requests()
    mixed, st, mon = _serve(L, reqs)
    assert st["finished"] == len(reqs)
    assert st["p50_s"] <= st["p99_s"] <= st["max_s"]
    for i, r in enumerate(reqs):
        alone, _, _ = _serve(L, [(r[0], 0.0) + tuple(r[2:])])
        assert rel_err(mixed[i], alone[0]) <= 1e-8, (i, rel_err(mixed[i], alone[0]))
    # oracle for a trip, a fault window and an event-free request
    for i in (0, 1, 3, 4):
        key, _, steps, kind, target, value, ev, ln = reqs[i]
        net = NETS[key][0]()
        nw = oemt.Network(net, DT, levels=NETS[key][1])
        events = []
        if kind == 0:
            events = [(ev, oemt.TRIP, target, 0.0)]
        elif kind == 1:
            events = [(ev, oemt.FAULT_ON, target, value), (ev + ln, oemt.FAULT_OFF, target, 0.0)]
        ref, _ = oemt.simulate(nw, steps, events, solver="dense", monitor=mon[key])
        assert rel_err(mixed[i], ref) <= 1e-8, (i, rel_err(mixed[i], ref))


def test_server_queues_when_slots_are_full(L):
    # 12 requests on a 4-slot network: later ones wait for slots and still finish correctly
    net = netgen.tile(1_000_000)
    srv = L.emt_server_create(25, 0)
    nid = L.emt_server_add_network(srv, net, DT, levels=2, max_slots=4, monitor=np.arange(8))
    rids = [L.emt_server_submit(srv, nid, 0.0, 60 + 5 * k) for k in range(12)]
    L.emt_server_run(srv)
    st = L.emt_server_stats(srv)
    assert st["finished"] == 12 and st["max_queue"] >= 8
    nw = oemt.Network(net, DT, levels=2)
    ref, _ = oemt.simulate(nw, 115, [], solver="dense", monitor=np.arange(8))
    for k, rid in enumerate(rids):
        got, times = L.emt_server_result(srv, rid)
        assert times[0] <= times[1] <= times[2]
        assert rel_err(got, ref[:60 + 5 * k]) <= 1e-8


def _oracle_run(net, levels, steps, kind, target, value, ev, ln, mon):
    nw = oemt.Network(net, DT, levels=levels)
    events = []
    if kind == 0:
        events = [(ev, oemt.TRIP, target, 0.0)]
    elif kind == 1:
        events = [(ev, oemt.FAULT_ON, target, value), (ev + ln, oemt.FAULT_OFF, target, 0.0)]
    ref, _ = oemt.simulate(nw, steps, events, solver="dense", monitor=mon)
    return ref


def test_server_private_networks_build_on_miss_and_hit_the_cache(L):
    # requests that bring their own networks: the first request of each network builds its store in
    # the admission path, a later request with the same content is served by the resident one
    base = netgen.tile(1_000_000)
    p1 = netgen.tile(1_000_007)
    p2 = netgen.tiled(1, 2, seed0=1_000_020)
    e1 = netgen.pick_branches(p1, 1, seed=5)
    mon1, mon2 = np.arange(0, p1["n_bus"], 13), np.arange(0, p2["n_bus"], 17)
    srv = L.emt_server_create(30, 0)
    nid = L.emt_server_add_network(srv, base, DT, levels=2, max_slots=8, monitor=np.arange(6))
    cases = [
        (p1, mon1, (0.00, 120, 0, int(e1[0]), 0.0, 50, 0)),
        (p1, mon1, (0.01, 90, 1, 9, 10.0, 20, 30)),
        (p2, mon2, (0.02, 100, -1, 0, 0.0, 0, 0)),
    ]
    rids = [L.emt_server_submit_network(srv, net, DT, *args, levels=2, monitor=mon) for net, mon, args in cases]
    rb = L.emt_server_submit(srv, nid, 0.0, 80)
    L.emt_server_run(srv)
    st = L.emt_server_stats(srv)
    assert st["finished"] == 4 and st["builds"] == 2 and st["cache_hits"] == 1 and st["evictions"] == 0
    assert st["build_s"] > 0
    for (net, mon, args), rid in zip(cases, rids):
        got, times = L.emt_server_result(srv, rid)
        assert times[0] <= times[1] <= times[2]
        ref = _oracle_run(net, 2, args[1], *args[2:], mon)
        assert rel_err(got, ref) <= 1e-8, rel_err(got, ref)
    got, _ = L.emt_server_result(srv, rb)
    assert rel_err(got, _oracle_run(base, 2, 80, -1, 0, 0.0, 0, 0, np.arange(6))) <= 1e-8


def test_server_evicts_idle_private_networks_under_the_budget(L):
    # a budget that holds one private network at a time: each arrival of the other network evicts
    # the idle one (least recently used) and builds its own
    p1 = netgen.tile(1_000_007)
    p2 = netgen.tiled(1, 2, seed0=1_000_020)
    mon1, mon2 = np.arange(5), np.arange(7)
    srv = L.emt_server_create(30, 120_000)
    r = [L.emt_server_submit_network(srv, p1, DT, 0.0, 60, levels=2, monitor=mon1),
         L.emt_server_submit_network(srv, p2, DT, 1.0, 60, levels=2, monitor=mon2),
         L.emt_server_submit_network(srv, p1, DT, 2.0, 60, levels=2, monitor=mon1)]
    L.emt_server_run(srv)
    st = L.emt_server_stats(srv)
    assert st["finished"] == 3 and st["builds"] == 3 and st["evictions"] == 2 and st["cache_hits"] == 0
    ref1 = _oracle_run(p1, 2, 60, -1, 0, 0.0, 0, 0, mon1)
    assert rel_err(L.emt_server_result(srv, r[0])[0], ref1) <= 1e-8
    assert rel_err(L.emt_server_result(srv, r[2])[0], ref1) <= 1e-8
    assert rel_err(L.emt_server_result(srv, r[1])[0], _oracle_run(p2, 2, 60, -1, 0, 0.0, 0, 0, mon2)) <= 1e-8


def test_server_random_private_networks_with_trips_and_faults_match_oracle(L):
    # private networks of irregular shape (hub, parallel branches, isolated buses): a trip of the
    # second of a parallel pair, a hub fault window, and a plain run, mixed on one server
    cases = []
    for seed in (31, 33):
        net = netgen.random_network(seed)
        a, b = np.asarray(net["br_a"]), np.asarray(net["br_b"])
        key = [(min(x, y), max(x, y)) for x, y in zip(a, b)]
        second = next(e for e in range(1, len(a)) if key[e] == key[0])
        hub = int(np.bincount(np.concatenate([a, b])).argmax())
        mon = np.arange(0, net["n_bus"], 9)
        cases += [(net, mon, (0.00, 110, 0, second, 0.0, 40, 0)),
                  (net, mon, (0.01, 90, 1, hub, 5.0, 20, 35)),
                  (net, mon, (0.02, 70, -1, 0, 0.0, 0, 0))]
    srv = L.emt_server_create(30, 0)
    rids = [L.emt_server_submit_network(srv, net, DT, *args, levels=3, monitor=mon) for net, mon, args in cases]
    L.emt_server_run(srv)
    st = L.emt_server_stats(srv)
    assert st["finished"] == len(cases) and st["builds"] == 2
    for (net, mon, args), rid in zip(cases, rids):
        got, _ = L.emt_server_result(srv, rid)
        ref = _oracle_run(net, 3, args[1], *args[2:], mon)
        assert rel_err(got, ref) <= 1e-8, rel_err(got, ref)
