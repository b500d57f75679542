"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs. Tolerances: 1e-10 for FP64 / float-float, 1e-8 for FP32
after refinement (relative to the max-norm of the reference)."""
import numpy as np
import pytest

import netgen
from oracle import dense as odense
from oracle import emt as oemt
from oracle import hinv as ohinv
from oracle import modify as omod
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = 50e-6
TOL = {0: 1e-10, 1: 1e-10, 2: 1e-8}


@pytest.fixture(scope="module")
def L():
    from paper_2105_10661_gb300 import buildlib
    buildlib.build()
    import paper_2105_10661_gb300._lib as lib
    assert torch.cuda.is_available()
    return lib


def _store_inputs(net):
    nw = oemt.Network(net, DT, want_tree=False)
    gr = nw.gr
    return nw, gr


def _apply(L, h, X):
    n, m = X.shape
    i_dev = torch.tensor(X.T.copy(), dtype=torch.float64, device="cuda")
    v_dev = torch.zeros_like(i_dev)
    L.emt_apply(h, i_dev, v_dev, nrhs=m, ld=n, max_refine=2 if h_prec(h) == 2 else 0)
    torch.cuda.synchronize()
    return v_dev.cpu().numpy().T


_PREC = {}


def h_prec(h):
    return _PREC.get(id(h), 0)


def _build(L, net_nw, levels=0, d_th=0, mode=0, prec=0):
    nw, gr = net_nw
    h = L.emt_build_hinv(gr["n_bus"], gr["frm"], gr["to"], gr["g"], levels=levels, d_th=d_th, mode=mode, precision=prec)
    _PREC[id(h)] = prec
    return h


def test_apply_rejects_a_tolerance_it_would_not_evaluate(L):
    nw, gr = _store_inputs(netgen.tile(1_000_000))
    h = _build(L, (nw, gr), levels=2, prec=2)
    i_dev = torch.ones(gr["n_bus"], dtype=torch.float64, device="cuda")
    v_dev = torch.zeros_like(i_dev)
    for tol in (1e-10, float("nan")):
        with pytest.raises(L.EmtError) as ex:
            L.emt_apply(h, i_dev, v_dev, max_refine=2, tol=tol)
        assert ex.value.code == L.EMT_ERR_UNSUPPORTED
    L.emt_apply(h, i_dev, v_dev, max_refine=2, tol=0.0)
    torch.cuda.synchronize()
    assert torch.isfinite(v_dev).all()


def _random_conductance_graph(seed):
    """A random multigraph with conductances and a shunt on every bus (so G is positive definite
    whatever is tripped): irregular trees, wide cuts at the hub, parallel branches."""
    n, a, b = netgen.random_multigraph(seed)
    rng = np.random.default_rng(seed + 100)
    g = rng.uniform(0.5, 20.0, len(a))
    frm = np.concatenate([a, np.arange(n, dtype=np.int32)])
    to = np.concatenate([b, np.full(n, -1, np.int32)])
    gv = np.concatenate([g, rng.uniform(0.01, 0.1, n)])
    G = np.zeros((n, n))
    for x, y, c in zip(frm, to, gv):
        G[x, x] += c
        if y >= 0:
            G[y, y] += c
            G[x, y] -= c
            G[y, x] -= c
    return n, frm, to, gv, G


@pytest.mark.parametrize("seed", [21, 22, 23])
@pytest.mark.parametrize("levels,d_th,prec", [(3, 0, 0), (0, 12, 0), (0, 12, 1), (4, 0, 2)])
def test_store_on_random_multigraph_matches_dense_solve_also_after_a_trip(L, seed, levels, d_th, prec):
    n, frm, to, gv, G = _random_conductance_graph(seed)
    h = L.emt_build_hinv(n, frm, to, gv, levels=levels, d_th=d_th, precision=prec)
    _PREC[id(h)] = prec
    X = np.random.default_rng(seed).standard_normal((n, 6))
    assert rel_err(_apply(L, h, X), odense.DenseSolver(G).solve(X)) <= TOL[prec]
    # trip the first of a parallel pair, then a hub branch whose pair of buses no earlier branch
    # joins (the store updates the first branch between two buses)
    first = {}
    for e in range(len(frm) - n):
        first.setdefault((min(frm[e], to[e]), max(frm[e], to[e])), e)
    hub_branches = [e for e in range(len(frm) - n - 12, len(frm) - n - 2)
                    if first[(min(frm[e], to[e]), max(frm[e], to[e]))] == e]
    for e in (0, hub_branches[0]):
        a, b, c = int(frm[e]), int(to[e]), float(gv[e])
        L.emt_modify_branch(h, a, b, -c)
        u = np.zeros(n)
        u[a] = 1.0
        u[b] -= 1.0
        G = G - c * np.outer(u, u)
        assert rel_err(_apply(L, h, X), odense.DenseSolver(G).solve(X)) <= TOL[prec], e


def test_hinv_get_partition_matches_tree_arrays(L):
    nw, gr = _store_inputs(netgen.tile(1_000_000))
    h = _build(L, (nw, gr), levels=2)
    perm, lo, hi, parent = L.emt_hinv_get_partition(h)
    t = h.tree()
    for k, a in (("perm", perm), ("lo", lo), ("hi", hi), ("parent", parent)):
        assert np.array_equal(a, t[k]), k
    assert np.array_equal(np.sort(perm), np.arange(gr["n_bus"]))
    assert lo[0] == 0 and hi[0] == gr["n_bus"] and parent[0] == -1


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("which,levels,d_th", [("tile", 2, 0), ("tiles8", 3, 0), ("small5", 2, 0), ("small37", 0, 7),
                                               ("small2", 1, 0), ("tile", 0, 20)])
def test_exact_apply_matches_dense_solve(L, prec, which, levels, d_th):
    if which == "tile":
        net = netgen.tile(1_000_000)
    elif which == "tiles8":
        net = netgen.tiled(2, 4)
    else:
        net = netgen.small_network(int(which[5:]), 91)
    ni = _store_inputs(net)
    h = _build(L, ni, levels, d_th, 0, prec)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((net["n_bus"], 3))
    got = _apply(L, h, X)
    ref = odense.DenseSolver(ni[0].G).solve(X)
    assert rel_err(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_paper_apply_matches_algorithm1(L, prec):
    net = netgen.tiled(2, 4)
    ni = _store_inputs(net)
    tree = __import__("oracle.partition", fromlist=["x"]).build_tree(net["n_bus"], net["br_a"], net["br_b"], 3)
    H = ohinv.HInv(ni[0].G, tree, ni[0].g_series, ohinv.PAPER)
    h = _build(L, ni, 3, 0, 1, prec)
    X = np.random.default_rng(6).standard_normal((net["n_bus"], 2))
    got = _apply(L, h, X)
    ref = H.apply(X)
    assert rel_err(got, ref) <= TOL[prec]


def test_paper_dth_sweep_matches_algorithm1_and_fig5_trend(L):
    # PAPER stores with leaves of at most d_th buses (levels 0): each equals the oracle's Algorithm 1
    # on the same tree, and the approximation error against the exact inverse falls as d_th grows,
    # to rounding at d_th = N (one leaf: the direct inverse), as in Fig. 5.
    net = netgen.tile(1_000_000)
    ni = _store_inputs(net)
    nw = ni[0]
    from oracle import partition as op
    X = np.random.default_rng(12).standard_normal((net["n_bus"], 3))
    exact = odense.DenseSolver(nw.G).solve(X)
    errs = []
    for d in (10, 45, 179):
        tree = op.build_tree(net["n_bus"], net["br_a"], net["br_b"], 0, d)
        H = ohinv.HInv(nw.G, tree, nw.g_series, ohinv.PAPER)
        h = _build(L, ni, 0, d, 1, 0)
        got = _apply(L, h, X)
        assert rel_err(got, H.apply(X)) <= 1e-10
        errs.append(rel_err(got, exact))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] <= 1e-12


def _branch_cases(nw, tree):
    from oracle import partition as op
    cross = int(tree["cut_e"][tree["cut_ptr"][0]])
    inner = None
    for e in range(len(nw.series_frm)):
        if op.leaf_of(tree, int(tree["pos"][nw.series_frm[e]])) == op.leaf_of(tree, int(tree["pos"][nw.series_to[e]])):
            inner = e
            break
    deep = None
    for p in range(1, len(tree["lo"])):
        if tree["left"][p] >= 0 and tree["cut_ptr"][p + 1] > tree["cut_ptr"][p]:
            deep = int(tree["cut_e"][tree["cut_ptr"][p]])
            break
    return [cross, inner, deep]


@pytest.mark.parametrize("prec", [0, 1])
def test_exact_modify_matches_recomputation(L, prec):
    net = netgen.tiled(2, 4)
    ni = _store_inputs(net)
    nw = ni[0]
    from oracle import partition as op
    tree = op.build_tree(net["n_bus"], net["br_a"], net["br_b"], 3)
    h = _build(L, ni, 3, 0, 0, prec)
    G = nw.G.copy()
    X = np.random.default_rng(7).standard_normal((net["n_bus"], 2))
    for e in _branch_cases(nw, tree):
        a, b, g = int(nw.series_frm[e]), int(nw.series_to[e]), float(nw.g_series[e])
        L.emt_modify_branch(h, a, b, -g)
        G = omod.modified_G(G, a, b, -g)
        assert rel_err(_apply(L, h, X), odense.DenseSolver(G).solve(X)) <= TOL[prec]
    # fault to ground and its removal
    L.emt_modify_branch(h, 11, -1, 0.1)
    G = omod.modified_G(G, 11, -1, 0.1)
    assert rel_err(_apply(L, h, X), odense.DenseSolver(G).solve(X)) <= TOL[prec]


def test_exact_modify_singular_rejected_and_store_unchanged(L):
    net = netgen.tile(1_000_000)
    ni = _store_inputs(net)
    h = _build(L, ni, 2, 0, 0, 0)
    X = np.random.default_rng(8).standard_normal((net["n_bus"], 1))
    before = _apply(L, h, X)
    a = int(ni[0].series_frm[3])
    with pytest.raises(L.EmtError) as e:
        L.emt_modify_branch(h, a, -1, -10.0 * ni[0].G[a, a])   # makes G indefinite
    assert e.value.code == L.EMT_ERR_SINGULAR
    after = _apply(L, h, X)
    assert np.array_equal(before, after)


def test_paper_modify_matches_algorithm2(L):
    net = netgen.tiled(2, 4)
    ni = _store_inputs(net)
    nw = ni[0]
    from oracle import partition as op
    tree = op.build_tree(net["n_bus"], net["br_a"], net["br_b"], 3)
    H = ohinv.HInv(nw.G, tree, nw.g_series, ohinv.PAPER)
    h = _build(L, ni, 3, 0, 1, 0)
    X = np.random.default_rng(9).standard_normal((net["n_bus"], 2))
    for e in _branch_cases(nw, tree):
        a, b, g = int(nw.series_frm[e]), int(nw.series_to[e]), float(nw.g_series[e])
        L.emt_modify_branch(h, a, b, -g)
        H = omod.algorithm2(H, nw.series_frm, nw.series_to, a, b, -g)
        assert rel_err(_apply(L, h, X), H.apply(X)) <= 1e-10


def _sim_compare(L, net, levels, steps, events, prec, mode=0, solver="dense", rpc=0, kernels=None):
    nw = oemt.Network(net, DT, levels=levels)
    oev = []
    for (st, kind, tgt, val) in events:
        oev.append((st, kind, tgt, val))
    ref, _ = oemt.simulate(nw, steps, oev, solver=solver)
    sim = L.emt_sim_create(net, DT, levels=levels, mode=mode, precision=prec)
    if kernels is not None:      # None: the launch shape emt_sim_create chose
        L.emt_sim_tune(sim, rpc, kernels)
    L.emt_sim_monitor(sim, np.arange(net["n_bus"]))
    for (st, kind, tgt, val) in events:
        L.emt_sim_schedule(sim, st, kind, tgt, val)
    rec = torch.zeros(steps, net["n_bus"], dtype=torch.float64, device="cuda")
    # two calls to exercise the step counter across emt_step calls
    h1 = steps // 2
    L.emt_step(sim, h1, rec[:h1])
    L.emt_step(sim, steps - h1, rec[h1:])
    torch.cuda.synchronize()
    final = L.emt_sim_read(sim, 0)
    got = rec.cpu().numpy()
    assert np.array_equal(final, got[-1])
    return rel_err(got, ref)


@pytest.mark.parametrize("kernels", [1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_sim_179_bus_trip_matches_oracle(L, prec, kernels):
    net = netgen.tile(1_000_000)
    e = netgen.pick_branch(net)
    err = _sim_compare(L, net, 2, 150, [(70, 0, e, 0.0)], prec, kernels=kernels)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("kernels", [1, 2, 3])
@pytest.mark.parametrize("rpc", [0, 7, 16, 64, 179])
def test_sim_fault_on_off_and_cta_shapes(L, rpc, kernels):
    net = netgen.tile(1_000_000)
    ev = [(30, 1, 17, 10.0), (90, 2, 17, 0.0), (100, 0, netgen.pick_branch(net), 0.0)]
    err = _sim_compare(L, net, 2, 140, ev, 1, rpc=rpc, kernels=kernels)
    assert err <= 1e-10, err


@pytest.mark.parametrize("kernels,rpc", [(1, 0), (2, 0), (3, 0), (4, 8), (4, 16)])
@pytest.mark.parametrize("prec", [0, 1])
def test_sim_changes_inside_fault_windows_match_oracle(L, prec, kernels, rpc):
    # a trip inside a fault window, overlapping faults at two buses, back-to-back and stacked
    # faults at one bus: clearing a fault takes back its own conductance only (Sec. IV), and the
    # oracle's trajectory for these orders is pinned by Kirchhoff's law at every bus and step
    from tests.test_oracle import _fault_event_sequences
    net = netgen.tile(1_000_000)
    for name, ev in _fault_event_sequences(net).items():
        err = _sim_compare(L, net, 2, 60, ev, prec, rpc=rpc, kernels=kernels)
        assert err <= TOL[prec], (name, err)


def test_sim_fault_cleared_where_none_is_on_is_rejected_before_stepping(L):
    net = netgen.tile(1_000_000)
    sim = L.emt_sim_create(net, DT, levels=2, precision=L.EMT_PREC_FF64)
    L.emt_sim_schedule(sim, 5, 1, 17, 10.0)
    L.emt_sim_schedule(sim, 8, 2, 18, 0.0)
    with pytest.raises(L.EmtError) as ex:
        L.emt_step(sim, 10)
    assert ex.value.code == L.EMT_ERR_STATE
    assert L.emt_sim_read(sim, 1)[0] == 0.0   # nothing was stepped


@pytest.mark.parametrize("cs", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("prec", [0, 1])
def test_sim_persistent_cluster_179_bus_events(L, prec, cs):
    # one cluster of cs CTAs runs the time loop; cs < 4 groups whole leaves, cs > 4 splits them
    net = netgen.tile(1_000_000)
    ev = [(30, 1, 17, 10.0), (90, 2, 17, 0.0), (100, 0, netgen.pick_branch(net), 0.0)]
    err = _sim_compare(L, net, 2, 140, ev, prec, rpc=cs, kernels=4)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", [0, 1])
def test_sim_persistent_cluster_1432_bus(L, prec):
    net = netgen.tiled(2, 4)
    e = netgen.pick_branch(net)
    err = _sim_compare(L, net, 3, 200, [(100, 0, e, 0.0)], prec, rpc=16, kernels=4)
    assert err <= TOL[prec], err


def test_sim_persistent_cluster_rejects_what_does_not_fit(L):
    # eight CTAs would each hold a whole 179-row leaf (258 KB): more than one CTA's shared memory
    sim = L.emt_sim_create(netgen.tiled(2, 4), DT, levels=3, precision=L.EMT_PREC_FF64)
    with pytest.raises(L.EmtError) as ex:
        L.emt_sim_tune(sim, 8, 4)
    assert ex.value.code == L.EMT_ERR_UNSUPPORTED
    sim32 = L.emt_sim_create(netgen.tile(1_000_000), DT, levels=2, precision=L.EMT_PREC_FP32)
    with pytest.raises(L.EmtError) as ex:
        L.emt_sim_tune(sim32, 1, 4)
    assert ex.value.code == L.EMT_ERR_UNSUPPORTED


@pytest.mark.parametrize("cs", [1, 4, 16])
def test_sim_persistent_cluster_ragged_network(L, cs):
    net = netgen.small_network(37, 5)
    err = _sim_compare(L, net, 3, 90, [(40, 0, 3, 0.0)], 1, rpc=cs, kernels=4)
    assert err <= 1e-10, err


def test_sim_paper_mode_matches_oracle_paper_stepping(L):
    net = netgen.tile(1_000_000)
    e = netgen.pick_branch(net)
    err = _sim_compare(L, net, 2, 120, [(60, 0, e, 0.0)], 1, mode=1, solver="paper")
    assert err <= 1e-10, err


@pytest.mark.parametrize("kernels", [1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_sim_1432_bus_matches_oracle(L, prec, kernels):
    net = netgen.tiled(2, 4)
    e = netgen.pick_branch(net)
    err = _sim_compare(L, net, 3, 200, [(100, 0, e, 0.0)], prec, kernels=kernels)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("net_name,levels", [("tile", 2), ("tiled", 3), ("small", 3)])
def test_sim_create_runs_the_persistent_kernel_by_default(L, net_name, levels):
    # no autotune: a fresh simulation runs generation 4 with the cluster the rule picks, launches
    # one kernel per stretch between events, and matches the oracle
    net = {"tile": lambda: netgen.tile(1_000_000), "tiled": lambda: netgen.tiled(2, 4),
           "small": lambda: netgen.small_network(37, 5)}[net_name]()
    sim = L.emt_sim_create(net, DT, levels=levels, precision=L.EMT_PREC_FF64)
    before = L.emt_sim_stats(sim)["launches"]
    L.emt_step(sim, 50)
    torch.cuda.synchronize()
    per_call = L.emt_sim_stats(sim)["launches"] - before
    assert per_call <= 4, per_call      # set-up, trig table, one persistent launch, advance
    e = netgen.pick_branch(net) if net_name != "small" else 3
    err = _sim_compare(L, net, levels, 80, [(40, 0, e, 0.0)], 1)
    assert err <= 1e-10, err


def test_sim_reset_reproduces_run_bit_for_bit(L):
    net = netgen.tiled(2, 4)
    e = netgen.pick_branch(net)
    sim = L.emt_sim_create(net, DT, levels=3, precision=L.EMT_PREC_FF64)
    L.emt_sim_schedule(sim, 50, 0, e)
    L.emt_sim_monitor(sim, np.arange(16))
    a = torch.zeros(100, 16, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    L.emt_step(sim, 100, a)
    L.emt_sim_reset(sim)
    L.emt_step(sim, 100, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_sim_ragged_small_network(L):
    net = netgen.small_network(37, 5)
    err = _sim_compare(L, net, 3, 90, [(40, 0, 3, 0.0)], 1)
    assert err <= 1e-10, err


def _random_network_trips(net):
    """Branches of a random network to trip: the second of the first parallel pair, and a hub
    branch whose buses no other branch joins."""
    a, b = np.asarray(net["br_a"]), np.asarray(net["br_b"])
    key = [(min(x, y), max(x, y)) for x, y in zip(a, b)]
    second = next(e for e in range(1, len(a)) if key[e] == key[0])
    count = {}
    for k in key:
        count[k] = count.get(k, 0) + 1
    hub = next(e for e in range(len(a) - 3, 0, -1) if count[key[e]] == 1)
    return second, hub


@pytest.mark.parametrize("seed", [31, 32, 33])
@pytest.mark.parametrize("prec,kernels", [(1, None), (1, 2), (0, 2), (2, 2)])
def test_sim_on_random_network_with_parallel_and_hub_trips_matches_oracle(L, seed, prec, kernels):
    net = netgen.random_network(seed)
    second, hub = _random_network_trips(net)
    hub_bus = int(np.bincount(np.concatenate([net["br_a"], net["br_b"]])).argmax())
    # a fault at the hub bus whose window holds both trips; a second fault at an isolated bus
    events = [(30, 1, hub_bus, 5.0), (35, 1, net["n_bus"] - 1, 2.0), (40, 0, second, 0.0), (70, 0, hub, 0.0),
              (85, 2, hub_bus, 0.0)]
    err = _sim_compare(L, net, 3, 110, events, prec, rpc=0, kernels=kernels)
    assert err <= TOL[prec], err


# ---------------------------------------------------------------- multi-column (N-1, scenarios)
def _msim_run(L, net, levels, steps, R, trips=None, src_scale=None, load_scale=None):
    sim = L.emt_sim_create(net, DT, levels=levels, nrhs=R, src_scale=src_scale, load_scale=load_scale)
    if trips:
        for c, (st, e) in trips.items():
            L.emt_sim_schedule(sim, st, 0, e, 0.0, c)
    L.emt_sim_monitor(sim, np.arange(net["n_bus"]))
    rec = torch.zeros(steps, R, net["n_bus"], dtype=torch.float64, device="cuda")
    h1 = steps // 3
    L.emt_step(sim, h1, rec[:h1])
    L.emt_step(sim, steps - h1, rec[h1:])
    torch.cuda.synchronize()
    final = L.emt_sim_read(sim, 0).reshape(R, net["n_bus"])
    got = rec.cpu().numpy()
    assert np.array_equal(final, got[-1])
    return got


@pytest.mark.parametrize("which,levels,R,steps", [("tile", 2, 8, 90), ("tiles8", 3, 12, 70)])
def test_multi_column_n1_trips_match_oracle(L, which, levels, R, steps):
    net = netgen.tile(1_000_000) if which == "tile" else netgen.tiled(2, 4)
    branches = netgen.pick_branches(net, R - 1, seed=11)
    trips = {c: (steps // 2 + (c % 3), int(branches[c])) for c in range(R - 1)}   # last column: no trip
    got = _msim_run(L, net, levels, steps, R, trips=trips)
    nw = oemt.Network(net, DT, levels=levels)
    worst = 0.0
    for c in range(R):
        ev = [(trips[c][0], oemt.TRIP, trips[c][1], 0.0)] if c in trips else []
        ref, _ = oemt.simulate(nw, steps, ev, solver="dense")
        worst = max(worst, rel_err(got[:, c, :], ref))
    assert worst <= 1e-8, worst


@pytest.mark.parametrize("seed", [31, 33])
def test_multi_column_on_random_network_with_parallel_and_hub_trips_matches_oracle(L, seed):
    net = netgen.random_network(seed)
    second, hub = _random_network_trips(net)
    R, steps, levels = 6, 80, 3
    trips = {0: (30, second), 1: (45, hub), 3: (30, hub)}   # columns 2, 4, 5: no trip
    got = _msim_run(L, net, levels, steps, R, trips=trips)
    nw = oemt.Network(net, DT, levels=levels)
    worst = 0.0
    for c in range(R):
        ev = [(trips[c][0], oemt.TRIP, trips[c][1], 0.0)] if c in trips else []
        ref, _ = oemt.simulate(nw, steps, ev, solver="dense")
        worst = max(worst, rel_err(got[:, c, :], ref))
    assert worst <= 1e-8, worst


def test_multi_column_scenarios_match_oracle(L):
    net = netgen.add_loads(netgen.tiled(2, 2), seed=13)
    R = 6
    ss, ls = netgen.scenario_scales(net, R, seed=13)
    got = _msim_run(L, net, 2, 60, R, src_scale=ss, load_scale=ls)
    nw = oemt.Network(net, DT, levels=2)
    worst = 0.0
    for c in range(R):
        ref, _ = oemt.simulate(nw, 60, [], solver="dense", src_scale=ss[c], load_scale=ls[c])
        worst = max(worst, rel_err(got[:, c, :], ref))
    assert worst <= 1e-8, worst


def test_multi_column_reset_and_unaligned_columns(L):
    net = netgen.tile(1_000_000)
    R = 5   # not a multiple of 4: scalar loads in the GEMM tail
    sim = L.emt_sim_create(net, DT, levels=2, nrhs=R)
    L.emt_sim_schedule(sim, 20, 0, 3, 0.0, 1)
    L.emt_sim_monitor(sim, np.arange(10))
    a = torch.zeros(40, R, 10, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    L.emt_step(sim, 40, a)
    L.emt_sim_reset(sim)
    L.emt_step(sim, 40, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    nw = oemt.Network(net, DT, levels=2)
    ref, _ = oemt.simulate(nw, 40, [(20, oemt.TRIP, 3, 0.0)], solver="dense", monitor=np.arange(10))
    assert rel_err(a[:, 1, :].cpu().numpy(), ref) <= 1e-8


@pytest.mark.parametrize("gemm", [1, 2, 3])
@pytest.mark.parametrize("which,levels,R,steps", [("tile", 2, 64, 50), ("tiles8", 3, 128, 40), ("tiles8", 3, 36, 30),
                                                   ("tiles8", 4, 100, 30)])
def test_multi_column_gemm_kinds_match_oracle(L, gemm, which, levels, R, steps):
    # gemm 1: FP32 CUDA-core products; 2: tcgen05 BF16x3 leaf GEMM (FP32 accumulate in TMEM), the
    # expansion by size (SIMT at these sizes); 3: tcgen05 leaf GEMM and expansion. 36 and 100
    # columns leave a ragged last 64-column tile; four levels give ancestor paths longer than one
    # 32-deep K chunk.
    net = netgen.tile(1_000_000) if which == "tile" else netgen.tiled(2, 4)
    branches = netgen.pick_branches(net, 3, seed=5)
    trips = {0: (steps // 2, int(branches[0])), R // 2: (steps // 3, int(branches[1])), R - 1: (5, int(branches[2]))}
    sim = L.emt_sim_create(net, DT, levels=levels, nrhs=R)
    L.emt_sim_tune(sim, 0, gemm)
    for c, (st, e) in trips.items():
        L.emt_sim_schedule(sim, st, 0, e, 0.0, c)
    mon = np.arange(0, net["n_bus"], 7)
    L.emt_sim_monitor(sim, mon)
    rec = torch.zeros(steps, R, len(mon), dtype=torch.float64, device="cuda")
    L.emt_step(sim, steps, rec)
    torch.cuda.synchronize()
    got = rec.cpu().numpy()
    nw = oemt.Network(net, DT, levels=levels)
    worst = 0.0
    for c in (0, 1, R // 2, R - 1):
        ev = [(trips[c][0], oemt.TRIP, trips[c][1], 0.0)] if c in trips else []
        ref, _ = oemt.simulate(nw, steps, ev, solver="dense", monitor=mon)
        worst = max(worst, rel_err(got[:, c, :], ref))
    assert worst <= 1e-8, worst


def test_bounded_wait_times_out_cleanly_and_context_survives(L):
    # a wait that nothing satisfies runs out after ~1 ms and reports EMT_ERR_TIMEOUT; the
    # context stays usable for the next call
    assert L.emt_selftest_bounded_wait(1000) == L.EMT_ERR_TIMEOUT
    net = netgen.tile(1_000_000)
    ni = _store_inputs(net)
    h = _build(L, ni, 2, 0, 0, 1)
    X = np.random.default_rng(3).standard_normal((net["n_bus"], 1))
    assert rel_err(_apply(L, h, X), odense.DenseSolver(ni[0].G).solve(X)) <= 1e-10


@pytest.mark.parametrize("tile,R", [(192, 200), (256, 128), (192, 64)])
def test_multi_column_leaf_tile_widths_match_oracle(L, tile, R):
    # leaf-GEMM tiles 192 or 256 columns wide (tensor memory rounded up to a power of two), with a
    # ragged or padded last column tile; tensor-core expansion on
    net = netgen.tiled(2, 4)
    steps = 30
    branches = netgen.pick_branches(net, 2, seed=9)
    trips = {1: (12, int(branches[0])), R - 1: (20, int(branches[1]))}
    sim = L.emt_sim_create(net, DT, levels=3, nrhs=R)
    L.emt_sim_tune(sim, tile, 3)
    for c, (st, e) in trips.items():
        L.emt_sim_schedule(sim, st, 0, e, 0.0, c)
    mon = np.arange(0, net["n_bus"], 9)
    L.emt_sim_monitor(sim, mon)
    rec = torch.zeros(steps, R, len(mon), dtype=torch.float64, device="cuda")
    L.emt_step(sim, steps, rec)
    torch.cuda.synchronize()
    got = rec.cpu().numpy()
    nw = oemt.Network(net, DT, levels=3)
    for c in (0, 1, R // 2, R - 1):
        ev = [(trips[c][0], oemt.TRIP, trips[c][1], 0.0)] if c in trips else []
        ref, _ = oemt.simulate(nw, steps, ev, solver="dense", monitor=mon)
        assert rel_err(got[:, c, :], ref) <= 1e-8, (c, rel_err(got[:, c, :], ref))


def test_multi_column_injection_variants_agree_and_match_oracle(L):
    # one column per thread, and two per thread with 6, 3 or 2 element ends per round trip (2, 3,
    # 4 CTAs per SM): the two-column variants batch the same arithmetic differently, bit for bit
    net = netgen.add_loads(netgen.tiled(2, 2), seed=13)
    R, steps = 64, 30
    ss, ls = netgen.scenario_scales(net, R, seed=13)
    branches = netgen.pick_branches(net, 2, seed=41)
    trips = {1: (10, int(branches[0])), R - 1: (18, int(branches[1]))}
    mon = np.arange(0, net["n_bus"], 9)
    out = {}
    for mode, ipp in ((1, 0), (2, 0), (3, 0), (4, 0), (4, 1), (2, 4), (1, 2)):
        sim = L.emt_sim_create(net, DT, levels=2, nrhs=R, src_scale=ss, load_scale=ls)
        L.emt_sim_set_inject(sim, mode, ipp)
        assert L.emt_sim_stats(sim)["inject_variant"] == mode
        for c, (st, e) in trips.items():
            L.emt_sim_schedule(sim, st, 0, e, 0.0, c)
        L.emt_sim_monitor(sim, mon)
        rec = torch.zeros(steps, R, len(mon), dtype=torch.float64, device="cuda")
        L.emt_step(sim, steps, rec)
        torch.cuda.synchronize()
        out[mode, ipp] = rec.cpu().numpy()
    for key in ((3, 0), (4, 0), (4, 1), (2, 4)):
        assert np.array_equal(out[2, 0], out[key]), key
    assert np.array_equal(out[1, 0], out[1, 2])
    out = {m: out[m, 0] for m in (1, 2)}
    nw = oemt.Network(net, DT, levels=2)
    for c in (0, 1, R - 1):
        ev = [(trips[c][0], oemt.TRIP, trips[c][1], 0.0)] if c in trips else []
        ref, _ = oemt.simulate(nw, steps, ev, solver="dense", monitor=mon, src_scale=ss[c], load_scale=ls[c])
        for mode in (1, 2):
            assert rel_err(out[mode][:, c, :], ref) <= 1e-8, (mode, c)
    odd = L.emt_sim_create(net, DT, levels=2, nrhs=5)
    with pytest.raises(L.EmtError) as e:
        L.emt_sim_set_inject(odd, 3)
    assert e.value.code == L.EMT_ERR_UNSUPPORTED


def test_multi_column_autotune_times_the_shapes_and_matches_oracle(L):
    # the autotuner times FP32 products and tcgen05 leaf tiles of every width, then the injection
    # kernel; the shape it keeps still matches the oracle, and a later simulation of the same shape
    # starts with it (bit-for-bit the same trajectory)
    net = netgen.tiled(2, 4)
    R, steps = 96, 30
    branches = netgen.pick_branches(net, 2, seed=21)
    trips = {3: (11, int(branches[0])), R - 2: (17, int(branches[1]))}
    mon = np.arange(0, net["n_bus"], 11)

    def make():
        sim = L.emt_sim_create(net, DT, levels=3, nrhs=R)
        for c, (st, e) in trips.items():
            L.emt_sim_schedule(sim, st, 0, e, 0.0, c)
        L.emt_sim_monitor(sim, mon)
        return sim

    def run(sim):
        rec = torch.zeros(steps, R, len(mon), dtype=torch.float64, device="cuda")
        L.emt_step(sim, steps, rec)
        torch.cuda.synchronize()
        return rec.cpu().numpy()

    sim = make()
    tn, kind = L.emt_sim_autotune(sim, 8)
    assert kind in (1, 2, 3) and tn in (0, 64, 128, 192, 256), (tn, kind)
    assert L.emt_sim_stats(sim)["inject_columns_per_thread"] in (1, 2)
    got = run(sim)
    nw = oemt.Network(net, DT, levels=3)
    for c in (0, 3, R // 2, R - 2):
        ev = [(trips[c][0], oemt.TRIP, trips[c][1], 0.0)] if c in trips else []
        ref, _ = oemt.simulate(nw, steps, ev, solver="dense", monitor=mon)
        assert rel_err(got[:, c, :], ref) <= 1e-8, (c, rel_err(got[:, c, :], ref))
    again = make()
    assert L.emt_sim_stats(again)["inject_columns_per_thread"] == L.emt_sim_stats(sim)["inject_columns_per_thread"]
    assert np.array_equal(run(again), got)


# ---------------------------------------------------------------- three-phase buses
def _three_phase(levels=3):
    from oracle import companion as ocm
    net = netgen.three_phase(netgen.tiled(1, 2))
    gr = ocm.three_phase_graph(net, DT)
    return net, gr, ocm.assemble_dense(gr)


@pytest.mark.parametrize("npb", [1, 3])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_three_phase_store_matches_dense_solve(L, prec, npb):
    # 358 buses, 1,074 nodes: mutual couplings enter as negative node branches; npb 3 partitions
    # by bus with block cuts (the default), npb 1 node by node
    net, gr, G = _three_phase()
    h = L.emt_build_hinv_from_network3(net, DT, levels=3, precision=prec, nodes_per_bus=npb)
    _PREC[id(h)] = prec
    X = np.random.default_rng(21).standard_normal((gr["n_bus"], 3))
    assert rel_err(_apply(L, h, X), odense.DenseSolver(G).solve(X)) <= TOL[prec]


@pytest.mark.parametrize("npb", [1, 3])
def test_three_phase_paper_store_matches_algorithm1(L, npb):
    # Algorithm 1's store is an approximation that depends on the tree and its cut columns: the
    # node-level tree, or the bus-level tree with block cuts
    from oracle import partition as op
    net, gr, G = _three_phase()
    ser = gr["to"] >= 0
    if npb == 1:
        tree = op.build_tree(gr["n_bus"], gr["frm"][ser], gr["to"][ser], 3)
        H = ohinv.HInv(G, tree, gr["g"][ser], ohinv.PAPER)
    else:
        tree = op.build_block_tree(gr["n_bus"], gr["frm"], gr["to"], 3, levels=3)
        H = ohinv.HInv(G, tree, gr["g"], ohinv.PAPER)
    h = L.emt_build_hinv_from_network3(net, DT, levels=3, mode=1, nodes_per_bus=npb)
    X = np.random.default_rng(22).standard_normal((gr["n_bus"], 2))
    assert rel_err(_apply(L, h, X), H.apply(X)) <= 1e-10


@pytest.mark.parametrize("npb,cut_line", [(1, False), (3, False), (3, True)])
def test_three_phase_line_trip_and_phase_fault_by_exact_node_updates(L, npb, cut_line):
    # a three-phase line trip removes Y (x) (e_a - e_b)(e_a - e_b)^T: fifteen exact rank-1 updates,
    # negative (cross-phase) branches first so that every intermediate G stays positive definite;
    # then a fault from one phase to ground. cut_line: a coupled line cut at the root, whose nine
    # phase-to-phase branches are the entries of one rank-3 block cut
    from oracle import companion as ocm
    net, gr, G = _three_phase()
    h = L.emt_build_hinv_from_network3(net, DT, levels=3, nodes_per_bus=npb)
    e = next(k for k in range(len(net["br_a"])) if net["kind"][k] == 0)
    if cut_line:
        t = h.tree()
        cut_buses = {(int(t["perm"][a]) // 3, int(t["perm"][b]) // 3)
                     for a, b in zip(t["cut_a"][t["cut_ptr"][0]:t["cut_ptr"][1]], t["cut_b"][t["cut_ptr"][0]:t["cut_ptr"][1]])}
        e = next(k for k in range(len(net["br_a"])) if net["kind"][k] == 0 and net["L_mut"][k] > 0 and
                 ((int(net["br_a"][k]), int(net["br_b"][k])) in cut_buses or
                  (int(net["br_b"][k]), int(net["br_a"][k])) in cut_buses))
    a, b = int(net["br_a"][e]), int(net["br_b"][e])
    Y = ocm.coupled_rl_admittance(float(net["R"][e]), float(net["L"][e]), float(net["L_mut"][e]), DT)
    cross = [(3 * a + p, 3 * b + q, Y[p, q]) for p in range(3) for q in range(3) if p != q]
    within = [(3 * x + p, 3 * x + q, -Y[p, q]) for x in (a, b) for p in range(3) for q in range(p + 1, 3)]
    self_ = [(3 * a + p, 3 * b + p, Y[p, p]) for p in range(3)]
    X = np.random.default_rng(23).standard_normal((gr["n_bus"], 2))
    for x, y, g in cross + within + self_:
        L.emt_modify_branch(h, x, y, -g)
        G = omod.modified_G(G, x, y, -g)
    assert rel_err(_apply(L, h, X), odense.DenseSolver(G).solve(X)) <= 1e-10
    node = 3 * int(net["br_a"][0]) + 1
    L.emt_modify_branch(h, node, -1, 0.1)
    G = omod.modified_G(G, node, -1, 0.1)
    assert rel_err(_apply(L, h, X), odense.DenseSolver(G).solve(X)) <= 1e-10


def test_block_paper_store_local_update_matches_algorithm2(L):
    # Algorithm 2 on a block store: a cross-phase branch of a line cut at the root changes one
    # entry of a block column; the GPU's literal Algorithm 2 equals the oracle's on the same tree
    from oracle import partition as op
    net, gr, G = _three_phase()
    tree = op.build_block_tree(gr["n_bus"], gr["frm"], gr["to"], 3, levels=3)
    H = ohinv.HInv(G, tree, gr["g"], ohinv.PAPER)
    h = L.emt_build_hinv_from_network3(net, DT, levels=3, mode=1)
    t = h.tree()
    assert np.array_equal(t["perm"], tree["perm"])
    # a cross-phase entry of a root block column that a coupled line fills
    a, b = next((int(t["perm"][t["cut_a"][c] + w]), int(t["perm"][t["cut_b"][c]]))
                for c in range(t["cut_ptr"][0], t["cut_ptr"][1]) for w in range(3)
                if (t["cut_a"][c] + w) % 3 != t["cut_b"][c] % 3
                and G[int(t["perm"][t["cut_a"][c] + w]), int(t["perm"][t["cut_b"][c]])] != 0.0)
    delta = 0.5 * float(G[a, b])
    L.emt_modify_branch(h, a, b, delta)
    H2 = omod.algorithm2(H, gr["frm"], gr["to"], a, b, delta)
    X = np.random.default_rng(26).standard_normal((gr["n_bus"], 2))
    assert rel_err(_apply(L, h, X), H2.apply(X)) <= 1e-10


def test_block_cuts_keep_buses_together_and_shrink_the_cut(L):
    # b buses per leaf become 3b nodes; a coupled line is one rank-3 cut instead of nine columns
    net, gr, G = _three_phase()
    hb = L.emt_build_hinv_from_network3(net, DT, levels=3)
    hn = L.emt_build_hinv_from_network3(net, DT, levels=3, nodes_per_bus=1)
    tb, tn = hb.tree(), hn.tree()
    assert np.array_equal(tb["perm"] % 3, np.tile(np.arange(3), len(tb["perm"]) // 3))
    assert np.all(tb["lo"] % 3 == 0) and np.all(tb["hi"] % 3 == 0)
    assert 3 * len(tb["cut_b"]) <= len(tn["cut_b"]) * 2
    X = np.random.default_rng(24).standard_normal((gr["n_bus"], 1))
    ref = odense.DenseSolver(G).solve(X)
    assert rel_err(_apply(L, hb, X), ref) <= 1e-10
    v = torch.zeros(gr["n_bus"], dtype=torch.float64, device="cuda")
    L.emt_apply_noalloc(hb, torch.tensor(X[:, 0], dtype=torch.float64, device="cuda"), v)
    torch.cuda.synchronize()
    assert rel_err(v.cpu().numpy(), ref[:, 0]) <= 1e-10


@pytest.mark.parametrize("prec,kernels", [(0, 1), (1, 1), (1, 2)])
def test_block_store_streaming_apply_matches_dense_solve(L, prec, kernels):
    # the streaming kernels (three, or the single launch) asked for on a small three-phase store:
    # the sweep matrix holds the block columns' factor rows combined with their coefficients
    net, gr, G = _three_phase()
    h = L.emt_build_hinv_from_network3(net, DT, levels=3, precision=prec)
    _PREC[id(h)] = prec
    assert L.emt_apply_tune(h, kernels) == 0   # planned by the first apply
    X = np.random.default_rng(25).standard_normal((gr["n_bus"], 2))
    ref = odense.DenseSolver(G).solve(X)
    assert rel_err(_apply(L, h, X), ref) <= TOL[prec]
    assert L.emt_apply_tune(h, kernels) == kernels
    # after an exact update of a cut entry the refreshed image still matches
    t = h.tree()
    a = int(t["perm"][t["cut_a"][0] + 1])
    b = int(t["perm"][t["cut_b"][0]])
    g = float(G[a, b])
    if g != 0.0:
        L.emt_modify_branch(h, a, b, 0.5 * g)
        G = omod.modified_G(G, a, b, 0.5 * g)
        assert rel_err(_apply(L, h, X), odense.DenseSolver(G).solve(X)) <= TOL[prec]


# ---------------------------------------------------------------- three-phase time stepping (NEXT-3)
def _sim3_run(L, net, levels, steps, trips, prec, monitor=None, halves=True, npb=0):
    sim = L.emt_sim3_create(net, DT, levels=levels, precision=prec, nodes_per_bus=npb)
    nn = 3 * net["n_bus"]
    mon = np.arange(nn) if monitor is None else np.asarray(monitor)
    L.emt_sim_monitor(sim, mon)
    for st, e in trips:
        L.emt_sim_schedule(sim, st, 0, e)
    rec = torch.zeros(steps, len(mon), dtype=torch.float64, device="cuda")
    h1 = steps // 2 if halves else steps
    L.emt_step(sim, h1, rec[:h1])
    if steps > h1:
        L.emt_step(sim, steps - h1, rec[h1:])
    torch.cuda.synchronize()
    return sim, rec.cpu().numpy()


@pytest.mark.parametrize("npb", [1, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_three_phase_stepping_matches_oracle_with_a_coupled_line_trip(L, prec, npb):
    # one tile in three phases with loads: coupled RL histories (3 x 3), RC branches per phase,
    # balanced sources and loads; the trip opens a coupled line at step 70 (15 exact node updates)
    from oracle import emt3 as oemt3
    net = netgen.three_phase(netgen.add_loads(netgen.tile(1_000_000), seed=3))
    e = next(k for k in range(len(net["br_a"])) if net["kind"][k] == 0 and net["L_mut"][k] > 0)
    ref, state = oemt3.simulate3(net, DT, 140, [(70, oemt3.TRIP, e, 0.0)])
    sim, got = _sim3_run(L, net, 2, 140, [(70, e)], prec, npb=npb)
    assert rel_err(got, ref) <= 1e-10, rel_err(got, ref)
    final = L.emt_sim_read(sim, 0)
    assert np.array_equal(final, got[-1])
    assert rel_err(final, state["v"]) <= 1e-10


def test_three_phase_stepping_1432_buses_matches_oracle(L):
    from oracle import emt3 as oemt3
    net = netgen.three_phase(netgen.tiled(2, 4))
    e = next(k for k in range(len(net["br_a"])) if net["kind"][k] == 0 and net["L_mut"][k] > 0)
    mon = np.sort(np.random.default_rng(17).choice(3 * net["n_bus"], 48, replace=False))
    ref, _ = oemt3.simulate3(net, DT, 90, [(40, oemt3.TRIP, e, 0.0)], monitor=mon)
    _, got = _sim3_run(L, net, 3, 90, [(40, e)], 1, monitor=mon)
    assert rel_err(got, ref) <= 1e-10, rel_err(got, ref)


@pytest.mark.parametrize("npb", [1, 3])
def test_three_phase_faults_and_a_trip_match_oracle(L, npb):
    # a phase-a fault at one bus, a three-phase fault (three node faults) at another overlapping it,
    # a coupled-line trip inside both windows; each clearing takes only its own fault back out
    from oracle import emt3 as oemt3
    net = netgen.three_phase(netgen.add_loads(netgen.tile(1_000_000), seed=3))
    e = next(k for k in range(len(net["br_a"])) if net["kind"][k] == 0 and net["L_mut"][k] > 0)
    ev = ([(30, oemt3.FAULT_ON, 3 * 17 + 0, 10.0)] + [(45, oemt3.FAULT_ON, 3 * 60 + p, 5.0) for p in range(3)]
          + [(55, oemt3.TRIP, e, 0.0), (70, oemt3.FAULT_OFF, 3 * 17 + 0, 0.0)]
          + [(90, oemt3.FAULT_OFF, 3 * 60 + p, 0.0) for p in range(3)])
    ref, _ = oemt3.simulate3(net, DT, 120, ev)
    sim = L.emt_sim3_create(net, DT, levels=2, precision=L.EMT_PREC_FF64, nodes_per_bus=npb)
    L.emt_sim_monitor(sim, np.arange(3 * net["n_bus"]))
    for st, kind, target, value in ev:
        L.emt_sim_schedule(sim, st, kind, target, value)
    rec = torch.zeros(120, 3 * net["n_bus"], dtype=torch.float64, device="cuda")
    L.emt_step(sim, 50, rec[:50])
    L.emt_step(sim, 70, rec[50:])
    torch.cuda.synchronize()
    assert rel_err(rec.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("seed,npb", [(31, 3), (33, 3)])
def test_three_phase_on_random_network_with_parallel_trip_and_faults_matches_oracle(L, seed, npb):
    # the random multigraph in three phases: wide cuts at the hub, parallel coupled lines (the
    # second of a pair trips), a second component and isolated buses, faults at the hub. Block cuts
    # only: node-level cuts at a hub of a third of the buses give cores of 2k in the thousands,
    # whose exact updates run for minutes in FP64 on one SM each
    from oracle import emt3 as oemt3
    net = netgen.three_phase(netgen.random_network(seed))
    second, _ = _random_network_trips(net)
    hub = int(np.bincount(np.concatenate([net["br_a"], net["br_b"]])).argmax())
    ev = ([(25, oemt3.FAULT_ON, 3 * hub + 1, 8.0), (40, oemt3.TRIP, second, 0.0),
           (60, oemt3.FAULT_OFF, 3 * hub + 1, 0.0)])
    ref, _ = oemt3.simulate3(net, DT, 90, ev)
    sim = L.emt_sim3_create(net, DT, levels=3, precision=L.EMT_PREC_FF64, nodes_per_bus=npb)
    L.emt_sim_monitor(sim, np.arange(3 * net["n_bus"]))
    for st, kind, target, value in ev:
        L.emt_sim_schedule(sim, st, kind, target, value)
    rec = torch.zeros(90, 3 * net["n_bus"], dtype=torch.float64, device="cuda")
    L.emt_step(sim, 90, rec)
    torch.cuda.synchronize()
    assert rel_err(rec.cpu().numpy(), ref) <= 1e-10, rel_err(rec.cpu().numpy(), ref)


@pytest.mark.parametrize("gemm", [1, 3])
def test_multi_column_gemm_kinds_on_random_network_match_oracle(L, gemm):
    net = netgen.random_network(32)
    second, hub = _random_network_trips(net)
    R, steps, levels = 36, 60, 4
    trips = {0: (20, second), 17: (30, hub), 35: (5, hub)}
    sim = L.emt_sim_create(net, DT, levels=levels, nrhs=R)
    L.emt_sim_tune(sim, 0, gemm)
    for c, (st, e) in trips.items():
        L.emt_sim_schedule(sim, st, 0, e, 0.0, c)
    mon = np.arange(0, net["n_bus"], 5)
    L.emt_sim_monitor(sim, mon)
    rec = torch.zeros(steps, R, len(mon), dtype=torch.float64, device="cuda")
    L.emt_step(sim, steps, rec)
    torch.cuda.synchronize()
    got = rec.cpu().numpy()
    nw = oemt.Network(net, DT, levels=levels)
    worst = 0.0
    for c in (0, 1, 17, 35):
        ev = [(trips[c][0], oemt.TRIP, trips[c][1], 0.0)] if c in trips else []
        ref, _ = oemt.simulate(nw, steps, ev, solver="dense", monitor=mon)
        worst = max(worst, rel_err(got[:, c, :], ref))
    assert worst <= 1e-8, worst


def test_three_phase_reset_repeats_and_rejects_other_events(L):
    net = netgen.three_phase(netgen.tile(1_000_000))
    sim = L.emt_sim3_create(net, DT, levels=2, precision=L.EMT_PREC_FF64)
    L.emt_sim_monitor(sim, np.arange(0, 3 * net["n_bus"], 7))
    L.emt_sim_schedule(sim, 30, 0, 3)
    with pytest.raises(L.EmtError) as ex:
        L.emt_sim_schedule(sim, 40, 1, 5, 10.0, column=3)
    assert ex.value.code == L.EMT_ERR_UNSUPPORTED
    with pytest.raises(L.EmtError) as ex:
        L.emt_sim_schedule(sim, 40, 1, 3 * net["n_bus"], 10.0)
    assert ex.value.code == L.EMT_ERR_INVALID
    bad = L.emt_sim3_create(net, DT, levels=2, precision=L.EMT_PREC_FF64)
    L.emt_sim_schedule(bad, 10, 2, 4)   # a clearing with no fault on: refused before any work
    with pytest.raises(L.EmtError) as ex:
        L.emt_step(bad, 20, None)
    assert ex.value.code == L.EMT_ERR_STATE
    a = torch.zeros(80, sim.n_mon, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    L.emt_step(sim, 80, a)
    L.emt_sim_reset(sim)
    L.emt_step(sim, 80, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    sim32 = None
    with pytest.raises(L.EmtError) as ex:
        sim32 = L.emt_sim3_create(net, DT, levels=2, precision=L.EMT_PREC_FP32)
    assert ex.value.code == L.EMT_ERR_UNSUPPORTED and sim32 is None
