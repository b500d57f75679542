"""Pins of the CPU oracle against facts fixed by the paper and by mathematics:
closed forms, hand-worked fixtures, identities the paper states, brute force
on small inputs. None of these re-types the oracle's own formula."""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import netgen
from oracle import companion as cm
from oracle import dense
from oracle import emt
from oracle import hinv
from oracle import modify
from oracle import partition as pt

GOLD = os.path.join(os.path.dirname(__file__), "golden")
DT = 50e-6


def _net(n_bus, seed, extra=None):
    return netgen.small_network(n_bus, seed, extra=extra)


# ---------------------------------------------------------------- companion models
def _rc_circuit(R, C, V):
    """One bus: a DC source V behind R (sine with f = 0, phase pi/2) and a shunt C."""
    return dict(n_bus=1, br_a=np.zeros(0, np.int32), br_b=np.zeros(0, np.int32), kind=np.zeros(0, np.int32),
                R=np.zeros(0), L=np.zeros(0), C=np.zeros(0), shunt_C=np.array([C]),
                src_bus=np.array([0], np.int32), src_Vm=np.array([V]), src_phi=np.array([np.pi / 2]),
                src_Rs=np.array([R]), load_bus=np.zeros(0, np.int32), load_amp=np.zeros(0),
                load_phi=np.zeros(0), freq=0.0)


def test_rc_charging_closed_form():
    # Trapezoidal charging from rest with the source switched on between 0 and dt:
    # v_n = V (1 - rho^(n-1) / (1 + a)),  rho = (1 - a)/(1 + a),  a = dt / (2RC)
    # (derived by hand from the trapezoidal rule; tends to V (1 - exp(-t/RC))).
    R, C, V, dt, n = 10.0, 20e-6, 1.7, 20e-6, 400
    nw = emt.Network(_rc_circuit(R, C, V), dt, want_tree=False)
    out, _ = emt.simulate(nw, n, solver="dense")
    a = dt / (2 * R * C)
    rho = (1 - a) / (1 + a)
    k = np.arange(1, n + 1)
    ref = V * (1 - rho ** (k - 1) / (1 + a))
    assert np.max(np.abs(out[:, 0] - ref)) <= 1e-13 * V
    analytic = V * (1 - np.exp(-k * dt / (R * C)))
    assert np.max(np.abs(out[:, 0] - analytic)) <= 2.0 * a * V   # O(dt) start-up offset only


def _phasor_check(kind):
    # Sine source (Rs) -> series branch (RL or RC) -> bus 1 with shunt C. The
    # trapezoidal steady state equals the phasor solution with s = j (2/dt) tan(w dt/2)
    # (the bilinear transform), so after the transient the samples match exactly.
    f, dt = 60.0, 50e-6
    w = 2 * np.pi * f
    Rs, R, L, Cs, Csh, V, phi = 1.0, 2.0, 10e-3, 50e-6, 100e-6, 1.3, 0.4
    net = dict(n_bus=2, br_a=np.array([0], np.int32), br_b=np.array([1], np.int32),
               kind=np.array([kind], np.int32), R=np.array([R]), L=np.array([L if kind == 0 else 0.0]),
               C=np.array([Cs if kind == 1 else 0.0]), shunt_C=np.array([20e-6, Csh]),
               src_bus=np.array([0], np.int32), src_Vm=np.array([V]), src_phi=np.array([phi]),
               src_Rs=np.array([Rs]), load_bus=np.zeros(0, np.int32), load_amp=np.zeros(0),
               load_phi=np.zeros(0), freq=f)
    nw = emt.Network(net, dt, want_tree=False)
    n = 8000
    out, _ = emt.simulate(nw, n, solver="dense")
    s = 1j * (2 / dt) * np.tan(w * dt / 2)
    Zb = R + (s * L if kind == 0 else 1 / (s * Cs))
    Y0 = 1 / Rs + s * 20e-6
    Y1 = s * Csh
    # nodal phasor equations
    A = np.array([[Y0 + 1 / Zb, -1 / Zb], [-1 / Zb, Y1 + 1 / Zb]])
    E = V * np.exp(1j * (phi - np.pi / 2)) / Rs     # sin(wt + phi) = Re(exp(j(wt + phi - pi/2)))
    Vp = np.linalg.solve(A, np.array([E, 0]))
    k = np.arange(n - 400, n + 1 - 1) + 1
    ref = np.real(Vp[None, :] * np.exp(1j * w * k * dt)[:, None])
    got = out[n - 400:]
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_rl_sine_steady_state_bilinear():
    _phasor_check(0)


def test_rc_series_sine_steady_state_bilinear():
    _phasor_check(1)


def test_kirchhoff_balance_every_step():
    net = netgen.tile(1_000_000)
    nw = emt.Network(net, DT, want_tree=False)
    el = nw.el
    n = net["n_bus"]
    Ih = np.zeros(len(el["g"]))
    active = np.ones(len(el["g"]), bool)
    sol = dense.DenseSolver(nw.G)
    w = 2 * np.pi * net["freq"]
    for step in range(1, 60):
        t = step * DT
        rhs = cm.source_injection(net, t) + cm.history_injection(el, Ih, n)
        v = sol.solve(rhs)
        cur, Ih = cm.update_history(el, v, Ih, active)
        # KCL: element currents leaving each bus + source currents (v - e)/Rs = 0
        bal = np.zeros(n)
        np.add.at(bal, el["a"], cur)
        m = el["b"] >= 0
        np.add.at(bal, el["b"][m], -cur[m])
        e = net["src_Vm"] * np.sin(w * t + net["src_phi"])
        np.add.at(bal, net["src_bus"], (v[net["src_bus"]] - e) / net["src_Rs"])
        scale = np.max(np.abs(cur)) + 1e-300
        assert np.max(np.abs(bal)) <= 1e-12 * max(scale, np.max(np.abs(net["src_Vm"] / net["src_Rs"])))


def _energy(nw, v, cur, active):
    net, el = nw.net, nw.el
    nb = el["n_series"]
    E = 0.5 * np.sum(net["shunt_C"] * v ** 2)
    ve = cm.branch_voltage(el, v)[:nb]
    for e in range(nb):
        if not active[e]:
            continue
        if net["kind"][e] == cm.KIND_RL:
            E += 0.5 * net["L"][e] * cur[e] ** 2
        else:
            vc = ve[e] - net["R"][e] * cur[e]
            E += 0.5 * net["C"][e] * vc ** 2
    return E


def test_passivity_sources_off():
    # With every source switched off, the trapezoidal energy never increases.
    net = _net(24, 5)
    nw = emt.Network(net, DT, want_tree=False)
    _, st = emt.simulate(nw, 200, solver="dense")
    off = dict(net)
    off["src_Vm"] = np.zeros_like(net["src_Vm"])
    nw2 = emt.Network(off, DT, want_tree=False)
    el = nw2.el
    Ih, active = st["Ih"].copy(), st["active"]
    v, cur = st["v"], st["cur"]
    sol = dense.DenseSolver(nw2.G)
    E_prev = _energy(nw2, v, cur, active)
    assert E_prev > 0
    for step in range(300):
        rhs = cm.history_injection(el, Ih, net["n_bus"])
        v = sol.solve(rhs)
        cur, Ih = cm.update_history(el, v, Ih, active)
        E = _energy(nw2, v, cur, active)
        assert E <= E_prev * (1 + 1e-12)
        E_prev = E


def test_lossless_lc_network_conserves_energy_exactly():
    # No resistance anywhere (R = 0, no Thevenin sources). For a linear system the trapezoidal rule
    # is the implicit midpoint rule, which keeps every quadratic invariant: once the driving current
    # sinks are zero at both ends of a step, the stored energy 1/2 C v^2 + 1/2 L i^2 stays the same
    # at every step. A wrong sign or coefficient in any history update breaks this at O(dt).
    base = _net(24, 5)
    net = dict(base)
    net["R"] = np.zeros_like(base["R"])
    net.update(src_bus=np.zeros(0, np.int32), src_Vm=np.zeros(0), src_phi=np.zeros(0), src_Rs=np.zeros(0),
               load_bus=np.array([0, 7, 13], np.int32), load_amp=np.array([0.1, 0.05, 0.08]),
               load_phi=np.array([0.0, 1.0, 2.0]))
    nw = emt.Network(net, DT, want_tree=False)
    el, n = nw.el, net["n_bus"]
    kinds = set(np.asarray(net["kind"]).tolist())
    assert cm.KIND_RL in kinds and cm.KIND_RC in kinds   # both series histories are exercised
    Ih = np.zeros(len(el["g"]))
    active = np.ones(len(el["g"]), bool)
    sol = dense.DenseSolver(nw.G)
    for step in range(1, 102):   # driven for 100 steps, then one step whose start still carries the sinks
        rhs = (cm.source_injection(net, step * DT) if step <= 100 else 0.0) + cm.history_injection(el, Ih, n)
        v = sol.solve(rhs)
        cur, Ih = cm.update_history(el, v, Ih, active)
    E0 = _energy(nw, v, cur, active)
    assert E0 > 0
    for _ in range(400):
        v = sol.solve(cm.history_injection(el, Ih, n))
        cur, Ih = cm.update_history(el, v, Ih, active)
        assert abs(_energy(nw, v, cur, active) - E0) <= 1e-11 * E0


# ---------------------------------------------------------------- exact solve
@pytest.mark.parametrize("n_bus", [2, 3, 5, 8, 13, 16])
def test_dense_inverse_brute_force(n_bus):
    nw = emt.Network(_net(n_bus, 100 + n_bus), DT, want_tree=False)
    Gi = dense.inverse(nw.G)
    assert np.allclose(Gi, np.linalg.inv(nw.G), rtol=1e-12, atol=0)
    assert np.max(np.abs(nw.G @ Gi - np.eye(n_bus))) <= 1e-12
    assert np.max(np.abs(Gi - Gi.T)) <= 1e-14 * np.max(np.abs(Gi))


def test_dense_matches_sparse_lu():
    # The paper's reference solver is LU based (Sec. V-C.1); SciPy's sparse LU agrees.
    net = netgen.tile(1_000_000)
    nw = emt.Network(net, DT, want_tree=False)
    rhs = np.random.default_rng(0).standard_normal(net["n_bus"])
    v1 = dense.DenseSolver(nw.G).solve(rhs)
    v2 = spla.splu(cm.assemble_sparse(nw.gr)).solve(rhs)
    assert np.max(np.abs(v1 - v2)) <= 1e-13 * np.max(np.abs(v1))


def test_two_bus_golden():
    gd = json.load(open(os.path.join(GOLD, "two_bus.json")))
    g0, g = gd["g0"], gd["g"]
    G = np.array([[g0 + g, -g], [-g, g0 + g]])
    tree = pt.build_tree(2, np.array([0]), np.array([1]), levels=1)
    gb = np.array([g])
    ex = hinv.HInv(G, tree, gb, hinv.EXACT).dense()
    pa = hinv.HInv(G, tree, gb, hinv.PAPER).dense()
    assert np.allclose(ex, gd["exact_inverse"], rtol=1e-15, atol=1e-16)
    assert np.allclose(pa, gd["paper_inverse"], rtol=1e-15, atol=1e-16)
    assert np.allclose(dense.inverse(G), gd["exact_inverse"], rtol=1e-15, atol=1e-16)


# ---------------------------------------------------------------- partition
def _graph_path(n):
    return np.arange(n - 1), np.arange(1, n)


def _graph_cycle(n):
    return np.arange(n), (np.arange(n) + 1) % n


def _graph_barbell(m):
    a, b = [], []
    for off in (0, m):
        for i in range(m):
            for j in range(i + 1, m):
                a.append(off + i); b.append(off + j)
    a.append(m - 1); b.append(m)
    return np.array(a), np.array(b)


def _graph_ladder(m):
    a, b = [], []
    for i in range(m):
        a.append(i); b.append(m + i)
        if i + 1 < m:
            a += [i, m + i]; b += [i + 1, m + i + 1]
    return np.array(a), np.array(b)


def _brute_min_bisection(n, a, b):
    import itertools
    best = None
    nA = (n + 1) // 2
    for S in itertools.combinations(range(n), nA):
        S = set(S)
        c = sum(1 for x, y in zip(a, b) if (x in S) != (y in S))
        best = c if best is None else min(best, c)
    return best


@pytest.mark.parametrize("name,graph,n", [
    ("path", _graph_path(11), 11), ("cycle", _graph_cycle(12), 12),
    ("barbell", _graph_barbell(6), 12), ("ladder", _graph_ladder(6), 12)])
def test_bisection_reaches_brute_force_minimum(name, graph, n):
    a, b = graph
    L, R = pt.bisect(np.arange(n), a, b)
    assert sorted(np.concatenate([L, R]).tolist()) == list(range(n))
    assert {len(L), len(R)} == {(n + 1) // 2, n // 2}
    assert pt.cut_size(L, R, a, b) == _brute_min_bisection(n, a, b)


def test_kl_never_worse_than_growth_and_small_brute_force():
    for seed in range(6):
        net = _net(12, 300 + seed, extra=6)
        a, b = net["br_a"], net["br_b"]
        L, R = pt.bisect(np.arange(12), a, b)
        best = _brute_min_bisection(12, a, b)
        assert pt.cut_size(L, R, a, b) >= best
        assert pt.cut_size(L, R, a, b) <= best + 2


def test_tree_invariants():
    net = netgen.tiled(2, 4)
    tr = pt.build_tree(net["n_bus"], net["br_a"], net["br_b"], levels=3)
    n = net["n_bus"]
    assert sorted(tr["perm"].tolist()) == list(range(n))
    assert len(tr["leaves"]) == 8
    assert [int(tr["hi"][j] - tr["lo"][j]) for j in tr["leaves"]] == [179] * 8
    for p in range(len(tr["lo"])):
        if tr["left"][p] >= 0:
            l, r = tr["left"][p], tr["right"][p]
            assert tr["lo"][l] == tr["lo"][p] and tr["hi"][l] == tr["lo"][r] and tr["hi"][r] == tr["hi"][p]
            assert tr["perm"][tr["lo"][l]:tr["hi"][l]].min() < tr["perm"][tr["lo"][r]:tr["hi"][r]].min()
            # the cut list is exactly the set of crossing branches
            Ls = set(tr["perm"][tr["lo"][l]:tr["hi"][l]].tolist())
            Rs = set(tr["perm"][tr["lo"][r]:tr["hi"][r]].tolist())
            cross = sorted(e for e, (x, y) in enumerate(zip(net["br_a"], net["br_b"]))
                           if (x in Ls and y in Rs) or (x in Rs and y in Ls))
            got = sorted(tr["cut_e"][tr["cut_ptr"][p]:tr["cut_ptr"][p + 1]].tolist())
            assert got == cross
            for c in range(tr["cut_ptr"][p], tr["cut_ptr"][p + 1]):
                assert tr["lo"][l] <= tr["cut_a"][c] < tr["hi"][l] <= tr["cut_b"][c] < tr["hi"][r]
    # leaf-size threshold reading: leaf iff size <= d_th
    tr2 = pt.build_tree(net["n_bus"], net["br_a"], net["br_b"], levels=0, d_th=100)
    for p in range(len(tr2["lo"])):
        size = tr2["hi"][p] - tr2["lo"][p]
        assert (tr2["left"][p] < 0) == (size <= 100)


def test_lca_brute_force():
    net = netgen.tiled(2, 2)
    tr = pt.build_tree(net["n_bus"], net["br_a"], net["br_b"], levels=0, d_th=20)
    rng = np.random.default_rng(3)
    leaves = tr["leaves"]
    for _ in range(200):
        u, v = rng.choice(leaves, 2)
        c = pt.lca(tr, int(u), int(v))
        # brute force: the deepest node whose range contains both leaves' ranges
        cands = [p for p in range(len(tr["lo"])) if tr["lo"][p] <= min(tr["lo"][u], tr["lo"][v])
                 and tr["hi"][p] >= max(tr["hi"][u], tr["hi"][v])]
        assert c == max(cands, key=lambda p: tr["depth"][p])


# ---------------------------------------------------------------- hierarchical inverse
@pytest.fixture(scope="module")
def tile_nw():
    return emt.Network(netgen.tile(1_000_000), DT, levels=2)


def test_exact_store_equals_dense_inverse(tile_nw):
    Gi = dense.inverse(tile_nw.G)
    H = hinv.HInv(tile_nw.G, tile_nw.tree, tile_nw.g_series, hinv.EXACT)
    assert hinv.relative_error(H.dense(), Gi) <= 1e-13
    x = np.random.default_rng(1).standard_normal(179)
    assert np.max(np.abs(H.apply(x) - Gi @ x)) <= 1e-13 * np.max(np.abs(Gi @ x))


@pytest.mark.parametrize("n_bus,levels", [(2, 1), (5, 2), (13, 3), (16, 2)])
def test_exact_store_tiny_brute_force(n_bus, levels):
    nw = emt.Network(_net(n_bus, 40 + n_bus), DT, levels=levels)
    H = hinv.HInv(nw.G, nw.tree, nw.g_series, hinv.EXACT)
    assert np.allclose(H.dense(), np.linalg.inv(nw.G), rtol=1e-11, atol=1e-14)


def test_paper_store_equals_dense_algorithm1(tile_nw):
    t = tile_nw.tree
    Gp = tile_nw.G[np.ix_(t["perm"], t["perm"])]
    A1 = hinv.algorithm1_dense(Gp, t)
    H = hinv.HInv(tile_nw.G, t, tile_nw.g_series, hinv.PAPER)
    assert np.max(np.abs(H.dense_node(0) - A1)) <= 1e-13 * np.max(np.abs(A1))


def test_eq5_offdiagonal_blocks_vanish(tile_nw):
    # Eq. 5 with M of Eq. 7: off-diagonal blocks 0, diagonal blocks I + M H^T and
    # I + M^T H. Those printed blocks are the blocks of Ginv G (the product order
    # is swapped in the text; G Ginv is its transpose, with blocks I + H M^T ...).
    # Algorithm 1 applies Eq. 4-7 at every node with G1, G2 the matrices whose
    # inverses the children hold (the true blocks when the children are leaves).
    t = tile_nw.tree
    H = hinv.HInv(tile_nw.G, t, tile_nw.g_series, hinv.PAPER)
    Gp = H.Gp
    checked_leaf_pair = False
    for p in range(len(t["lo"])):
        if t["left"][p] < 0:
            continue
        l, r = int(t["left"][p]), int(t["right"][p])
        lo, hi = int(t["lo"][p]), int(t["hi"][p])
        ml = int(t["hi"][l] - lo)
        Gi = H.dense_node(p)
        if t["left"][l] < 0 and t["left"][r] < 0:
            G1, G2 = Gp[lo:lo + ml, lo:lo + ml], Gp[lo + ml:hi, lo + ml:hi]
            checked_leaf_pair = True
        else:
            G1, G2 = np.linalg.inv(H.dense_node(l)), np.linalg.inv(H.dense_node(r))
        Hm = Gp[lo:hi, lo:hi][:ml, ml:]
        Gblk = np.block([[G1, Hm], [Hm.T, G2]])
        prod = Gi @ Gblk
        M = Gi[:ml, ml:]
        scale = np.max(np.abs(prod))
        assert np.max(np.abs(Gblk @ Gi - prod.T)) <= 1e-12 * scale
        assert np.max(np.abs(prod[:ml, ml:])) <= 1e-12 * scale
        assert np.max(np.abs(prod[ml:, :ml])) <= 1e-12 * scale
        assert np.max(np.abs(prod[:ml, :ml] - (np.eye(ml) + M @ Hm.T))) <= 1e-12 * scale
        assert np.max(np.abs(prod[ml:, ml:] - (np.eye(hi - lo - ml) + M.T @ Hm))) <= 1e-12 * scale
    assert checked_leaf_pair


def test_eq9_low_rank_form_equals_eq7(tile_nw):
    t = tile_nw.tree
    H = hinv.HInv(tile_nw.G, t, tile_nw.g_series, hinv.PAPER)
    p = 0
    l, r = int(t["left"][p]), int(t["right"][p])
    A, B = H.dense_node(l), H.dense_node(r)
    lo, hi = int(t["lo"][p]), int(t["hi"][p])
    ml = int(t["hi"][l] - lo)
    Hm = H.Gp[lo:hi, lo:hi][:ml, ml:]
    M7 = -A @ Hm @ B
    M9 = -(H.P[p]) @ H.Q[p].T
    assert np.max(np.abs(M7 - M9)) <= 1e-14 * np.max(np.abs(M7))
    hl, hr = H.cut_columns(p)
    assert np.array_equal(hl @ hr.T, Hm)


def test_no_coupling_paper_equals_exact():
    # Two disconnected halves: H = 0, so the approximation is exact.
    net = netgen.small_network(10, 9)
    a, b = net["br_a"], net["br_b"]
    keep = ~(((a < 5) & (b >= 5)) | ((a >= 5) & (b < 5)))
    for k in ("br_a", "br_b", "kind", "R", "L", "C"):
        net[k] = net[k][keep]
    nw = emt.Network(net, DT, levels=1)
    ex = hinv.HInv(nw.G, nw.tree, nw.g_series, hinv.EXACT).dense()
    pa = hinv.HInv(nw.G, nw.tree, nw.g_series, hinv.PAPER).dense()
    assert np.max(np.abs(ex - pa)) <= 1e-15 * np.max(np.abs(ex))


def test_paper_error_falls_as_threshold_grows():
    # Fig. 5: the approximation error drops as d_th grows, to zero at d_th = N.
    nw = emt.Network(netgen.tile(1_000_000), DT, want_tree=False)
    Gi = dense.inverse(nw.G)
    errs = []
    for d in (10, 45, 179):
        tr = pt.build_tree(179, nw.series_frm, nw.series_to, 0, d)
        errs.append(hinv.relative_error(hinv.HInv(nw.G, tr, nw.g_series, hinv.PAPER).dense(), Gi))
    assert errs[0] >= errs[1] and errs[2] <= 1e-14


# ---------------------------------------------------------------- modification
def test_sherman_morrison_and_woodbury_closed_forms(tile_nw):
    G = tile_nw.G
    Gi = dense.inverse(G)
    a, b = int(tile_nw.series_frm[7]), int(tile_nw.series_to[7])
    g = float(tile_nw.g_series[7])
    u = modify.u_vector(179, a, b)
    G2 = modify.modified_G(G, a, b, -g)
    assert np.max(np.abs(dense.sherman_morrison(Gi, u, -g) - np.linalg.inv(G2))) <= 1e-12 * np.max(np.abs(Gi))
    a2, b2 = int(tile_nw.series_frm[50]), int(tile_nw.series_to[50])
    g2 = float(tile_nw.g_series[50])
    U = np.stack([u, modify.u_vector(179, a2, b2)], axis=1)
    G3 = modify.modified_G(G2, a2, b2, -g2)
    assert np.max(np.abs(dense.woodbury(Gi, U, [-g, -g2]) - np.linalg.inv(G3))) <= 1e-12 * np.max(np.abs(Gi))


def _cross_and_inner_branches(nw):
    t = nw.tree
    cross = int(t["cut_e"][t["cut_ptr"][0]])
    inner = None
    for e in range(len(nw.series_frm)):
        la = pt.leaf_of(t, int(t["pos"][nw.series_frm[e]]))
        lb = pt.leaf_of(t, int(t["pos"][nw.series_to[e]]))
        if la == lb:
            inner = e
            break
    return cross, inner


def test_exact_rebuild_after_trip_equals_dense(tile_nw):
    H = hinv.HInv(tile_nw.G, tile_nw.tree, tile_nw.g_series, hinv.EXACT)
    for e in _cross_and_inner_branches(tile_nw):
        a, b, g = int(tile_nw.series_frm[e]), int(tile_nw.series_to[e]), float(tile_nw.g_series[e])
        H2 = modify.rebuild(H, tile_nw.series_frm, tile_nw.series_to, a, b, -g)
        ref = np.linalg.inv(modify.modified_G(tile_nw.G, a, b, -g))
        assert hinv.relative_error(H2.dense(), ref) <= 1e-13


def test_algorithm2_to_root_equals_rebuild(tile_nw):
    H = hinv.HInv(tile_nw.G, tile_nw.tree, tile_nw.g_series, hinv.PAPER)
    for e in _cross_and_inner_branches(tile_nw):
        a, b, g = int(tile_nw.series_frm[e]), int(tile_nw.series_to[e]), float(tile_nw.g_series[e])
        A = modify.algorithm2(H, tile_nw.series_frm, tile_nw.series_to, a, b, -g, to_root=True)
        R = modify.rebuild(H, tile_nw.series_frm, tile_nw.series_to, a, b, -g)
        assert np.array_equal(A.dense(), R.dense())


def test_algorithm2_literal_touches_only_local_blocks(tile_nw):
    # Fault to ground inside one leaf: the LCA is the leaf itself, so only that
    # leaf's inverse changes (Sec. IV-A, best case), and it is the direct inverse
    # of the modified leaf block.
    t = tile_nw.tree
    H = hinv.HInv(tile_nw.G, t, tile_nw.g_series, hinv.PAPER)
    bus = int(t["perm"][3])
    A = modify.algorithm2(H, tile_nw.series_frm, tile_nw.series_to, bus, -1, 0.1)
    j = pt.leaf_of(t, 3)
    lo, hi = int(t["lo"][j]), int(t["hi"][j])
    blk = modify.modified_G(tile_nw.G, bus, -1, 0.1)[np.ix_(t["perm"][lo:hi], t["perm"][lo:hi])]
    assert np.allclose(A.leaf_inv[j], np.linalg.inv(blk), rtol=1e-12, atol=1e-15)
    for p in A.P:
        assert np.array_equal(A.P[p], H.P[p]) and np.array_equal(A.Q[p], H.Q[p])
    for q in A.leaf_inv:
        if q != j:
            assert np.array_equal(A.leaf_inv[q], H.leaf_inv[q])
    # with the LCA at the root, the literal algorithm is a full rebuild
    e = int(t["cut_e"][t["cut_ptr"][0]])
    a, b, g = int(tile_nw.series_frm[e]), int(tile_nw.series_to[e]), float(tile_nw.g_series[e])
    L = modify.algorithm2(H, tile_nw.series_frm, tile_nw.series_to, a, b, -g)
    R = modify.rebuild(H, tile_nw.series_frm, tile_nw.series_to, a, b, -g)
    assert np.array_equal(L.dense(), R.dense())


def test_modification_saving_golden():
    gd = json.load(open(os.path.join(GOLD, "paper_numbers.json")))["modification_saving"]
    assert round(100 * modify.leaf_inversion_saving(gd["d_th"], gd["n"]), 1) == gd["printed_percent"]


# ---------------------------------------------------------------- stepping
def test_stepping_solvers_agree_with_trip_and_fault():
    net = netgen.tile(1_000_000)
    nw = emt.Network(net, DT, levels=2)
    e = netgen.pick_branch(net)
    ev = [(30, emt.TRIP, e, 0.0), (40, emt.FAULT_ON, 17, 10.0), (55, emt.FAULT_OFF, 17, 0.0)]
    d, sd = emt.simulate(nw, 80, ev, solver="dense")
    x, sx = emt.simulate(nw, 80, ev, solver="exact")
    assert np.max(np.abs(d - x)) <= 1e-11 * np.max(np.abs(d))
    assert sd["cur"][e] == 0.0 and sd["Ih"][e] == 0.0
    p, _ = emt.simulate(nw, 80, ev, solver="paper")
    assert np.all(np.isfinite(p))


def _fault_event_sequences(net):
    """Event orders in which one change happens while a fault is on (steps, kind, target, value)."""
    e = netgen.pick_branch(net)
    e17 = next(i for i in range(len(net["br_a"])) if 17 in (int(net["br_a"][i]), int(net["br_b"][i])))
    return {
        "trip inside a fault window": [(20, emt.FAULT_ON, 17, 10.0), (30, emt.TRIP, e, 0.0),
                                       (40, emt.FAULT_OFF, 17, 0.0)],
        "trip at the faulted bus inside its window": [(20, emt.FAULT_ON, 17, 10.0), (28, emt.TRIP, e17, 0.0),
                                                      (41, emt.FAULT_OFF, 17, 0.0)],
        "overlapping faults at two buses": [(20, emt.FAULT_ON, 17, 10.0), (25, emt.FAULT_ON, 60, 5.0),
                                            (35, emt.FAULT_OFF, 17, 0.0), (45, emt.FAULT_OFF, 60, 0.0)],
        "back-to-back and stacked faults at one bus": [
            (20, emt.FAULT_ON, 17, 10.0), (30, emt.FAULT_OFF, 17, 0.0), (30, emt.FAULT_ON, 17, 4.0),
            (33, emt.FAULT_ON, 17, 20.0), (38, emt.FAULT_OFF, 17, 0.0), (45, emt.FAULT_OFF, 17, 0.0)],
    }


def _kirchhoff_through_events(nw, nsteps, events, solver):
    # Kirchhoff's current law at every bus and step, for the network the events describe: a
    # tripped branch carries nothing from its trip on, and each fault that is on draws v_a / R_f
    # (faults at one bus clear in the order they came on). The voltages come from the oracle's
    # stepping; the element currents follow from them by the companion models.
    out, _ = emt.simulate(nw, nsteps, events, solver=solver)
    net, el = nw.net, nw.el
    n = net["n_bus"]
    w = 2 * np.pi * net["freq"]
    Ih = np.zeros(len(el["g"]))
    active = np.ones(len(el["g"]), bool)
    on = {}
    worst = 0.0
    for s in range(nsteps):
        step = s + 1
        for (st, kind, tgt, val) in events:
            if st != step:
                continue
            if kind == emt.TRIP:
                active[tgt] = False
                Ih[tgt] = 0.0
            elif kind == emt.FAULT_ON:
                on.setdefault(tgt, []).append(val)
            else:
                on[tgt].pop(0)
        v = out[s]
        cur, Ih = cm.update_history(el, v, Ih, active)
        bal = np.zeros(n)
        np.add.at(bal, el["a"], cur)
        m = el["b"] >= 0
        np.add.at(bal, el["b"][m], -cur[m])
        e = net["src_Vm"] * np.sin(w * step * nw.dt + net["src_phi"])
        np.add.at(bal, net["src_bus"], (v[net["src_bus"]] - e) / net["src_Rs"])
        for bus, rs in on.items():
            bal[bus] += sum(v[bus] / r for r in rs)
        scale = max(np.max(np.abs(cur)), np.max(np.abs(net["src_Vm"] / net["src_Rs"])))
        worst = max(worst, np.max(np.abs(bal)) / scale)
    return worst


@pytest.mark.parametrize("solver", ["dense", "exact"])
def test_kirchhoff_balance_through_trips_and_overlapping_faults(solver):
    net = netgen.tile(1_000_000)
    nw = emt.Network(net, DT, levels=2)
    for name, ev in _fault_event_sequences(net).items():
        assert _kirchhoff_through_events(nw, 55, ev, solver) <= 1e-12, name


def test_fault_cleared_where_none_is_on_is_rejected():
    nw = emt.Network(netgen.tile(1_000_000), DT, want_tree=False)
    with pytest.raises(ValueError):
        emt.simulate(nw, 10, [(3, emt.FAULT_ON, 17, 10.0), (5, emt.FAULT_OFF, 18, 0.0)])


# ---------------------------------------------------------------- three-phase buses (3 nodes per bus)
def test_coupled_rl_admittance_closed_form():
    # (R I + (2/dt)(L I + M (J - I)))^-1 = (alpha - beta)^-1 (I - beta / (alpha + 2 beta) J),
    # alpha = R + 2L/dt, beta = 2M/dt (eigenvalues alpha + 2 beta on (1,1,1), alpha - beta twice);
    # M = 0 gives the single-phase companion conductance on the diagonal
    R, L, M, dt = 1.3, 0.021, 0.006, 50e-6
    al, be = R + 2 * L / dt, 2 * M / dt
    J = np.ones((3, 3))
    closed = (np.eye(3) - be / (al + 2 * be) * J) / (al - be)
    assert np.allclose(cm.coupled_rl_admittance(R, L, M, dt), closed, rtol=1e-13, atol=0)
    assert np.allclose(cm.coupled_rl_admittance(R, L, 0.0, dt), np.eye(3) / al, rtol=1e-14, atol=0)
    Y = cm.coupled_rl_admittance(R, L, M, dt)
    assert np.all(np.linalg.eigvalsh(Y) > 0) and np.all(Y[~np.eye(3, dtype=bool)] < 0)


def _block_assembly(net, dt):
    # the same G from 3 x 3 blocks: Y at (a, a) and (b, b), -Y at (a, b) and (b, a)
    n = net["n_bus"]
    G = np.zeros((3 * n, 3 * n))
    for e in range(len(net["br_a"])):
        a, b = int(net["br_a"][e]), int(net["br_b"][e])
        if net["kind"][e] == 0:
            Y = cm.coupled_rl_admittance(float(net["R"][e]), float(net["L"][e]), float(net["L_mut"][e]), dt)
        else:
            Y = np.eye(3) / (float(net["R"][e]) + dt / (2 * float(net["C"][e])))
        for (x, y, s) in ((a, a, 1.0), (b, b, 1.0), (a, b, -1.0), (b, a, -1.0)):
            G[3 * x:3 * x + 3, 3 * y:3 * y + 3] += s * Y
    for i in range(n):
        G[3 * i:3 * i + 3, 3 * i:3 * i + 3] += np.eye(3) * 2 * float(net["shunt_C"][i]) / dt
    for k in range(len(net["src_bus"])):
        i = int(net["src_bus"][k])
        G[3 * i:3 * i + 3, 3 * i:3 * i + 3] += np.eye(3) / float(net["src_Rs"][k])
    return G


def test_three_phase_node_branches_equal_block_assembly():
    net = netgen.three_phase(netgen.small_network(13, 77))
    gr = cm.three_phase_graph(net, DT)
    G = cm.assemble_dense(gr)
    Gb = _block_assembly(net, DT)
    assert np.allclose(G, Gb, rtol=0, atol=1e-12 * np.abs(Gb).max())
    assert np.allclose(G, G.T) and np.linalg.eigvalsh(G).min() > 0
    assert (gr["g"] < 0).any()   # the mutual couplings appear as negative node branches


def test_three_phase_without_mutual_is_three_decoupled_copies():
    net = netgen.small_network(13, 77)
    net3 = netgen.three_phase(net)
    net3["L_mut"] = np.zeros(len(net["br_a"]))
    G3 = cm.assemble_dense(cm.three_phase_graph(net3, DT))
    G1 = cm.assemble_dense(cm.graph(net, DT))
    assert np.allclose(G3, np.kron(G1, np.eye(3)), rtol=1e-14, atol=0)


def test_three_phase_exact_store_equals_dense_inverse():
    # the hierarchical store holds the node graph with its negative (mutual) branches exactly
    net = netgen.three_phase(netgen.tile(1_000_000))
    gr = cm.three_phase_graph(net, DT)
    G = cm.assemble_dense(gr)
    ser = gr["to"] >= 0
    tree = pt.build_tree(gr["n_bus"], gr["frm"][ser], gr["to"][ser], levels=2)
    H = hinv.HInv(G, tree, gr["g"][ser], hinv.EXACT)
    X = np.random.default_rng(3).standard_normal((gr["n_bus"], 2))
    assert np.allclose(H.apply(X), np.linalg.solve(G, X), rtol=0, atol=1e-12 * np.abs(np.linalg.solve(G, X)).max())


def _block_case(levels=2):
    net = netgen.three_phase(netgen.tile(1_000_000))
    gr = cm.three_phase_graph(net, DT)
    return net, gr, cm.assemble_dense(gr), pt.build_block_tree(gr["n_bus"], gr["frm"], gr["to"], 3, levels=levels)


def test_block_tree_keeps_buses_together_and_factors_each_h_exactly():
    # Eq. 3: H is the off-diagonal block G_lr; with block cuts h_l h_r^T must equal it entry for
    # entry, every node must hold whole buses (b buses -> 3b nodes), and a coupled line costs one
    # rank-3 cut instead of one column per node branch
    net, gr, G, tb = _block_case()
    n = gr["n_bus"]
    perm = tb["perm"]
    assert np.array_equal(perm % 3, np.tile(np.arange(3), n // 3))
    assert np.array_equal(perm[0::3] // 3, perm[1::3] // 3) and np.array_equal(perm[0::3] // 3, perm[2::3] // 3)
    assert np.all(tb["lo"] % 3 == 0) and np.all(tb["hi"] % 3 == 0)
    st = hinv.HInv(G, tb, np.zeros(0), hinv.EXACT)
    Gp = G[np.ix_(perm, perm)]
    pairs_total = 0
    for p in range(len(tb["lo"])):
        l, r = int(tb["left"][p]), int(tb["right"][p])
        if l < 0:
            continue
        hl, hr = st.cut_columns(p)
        H = Gp[tb["lo"][l]:tb["hi"][l], tb["lo"][r]:tb["hi"][r]]
        assert np.array_equal(hl @ hr.T, H)
        # bus pairs joined across this cut, counted by brute force from the series branches
        lb = set(int(x) for x in perm[tb["lo"][l]:tb["hi"][l]] // 3)
        rb = set(int(x) for x in perm[tb["lo"][r]:tb["hi"][r]] // 3)
        pairs = {(min(a, b), max(a, b)) for a, b in zip(net["br_a"], net["br_b"])
                 if (a in lb and b in rb) or (a in rb and b in lb)}
        assert tb["cut_ptr"][p + 1] - tb["cut_ptr"][p] == 3 * len(pairs)
        pairs_total += len(pairs)
    ser = gr["to"] >= 0
    tn = pt.build_tree(n, gr["frm"][ser], gr["to"][ser], levels=2)
    assert len(tb["cut_b"]) == 3 * pairs_total < len(tn["cut_b"])


def test_block_store_is_the_exact_inverse_and_paper_store_is_algorithm1():
    net, gr, G, tb = _block_case(levels=3)
    perm = tb["perm"]
    ex = hinv.HInv(G, tb, np.zeros(0), hinv.EXACT)
    Ginv = np.linalg.inv(G)
    assert hinv.relative_error(ex.dense(), Ginv) <= 1e-12
    pa = hinv.HInv(G, tb, np.zeros(0), hinv.PAPER)
    ref = hinv.algorithm1_dense(G[np.ix_(perm, perm)], tb)
    got = pa.dense()[np.ix_(perm, perm)]
    assert hinv.relative_error(got, ref) <= 1e-12


def test_block_store_local_update_equals_rebuild():
    # Sec. IV on a block store: a cross-phase node branch of a cut line changes its column's
    # coefficient (read from G), and Algorithm 2 carried to the root equals a rebuild
    net, gr, G, tb = _block_case()
    st = hinv.HInv(G, tb, gr["g"], hinv.EXACT)
    p = 0
    a = int(tb["cut_a"][3 * tb["cut_ptr"][p] + 1])
    y = int(tb["cut_b"][tb["cut_ptr"][p]])
    xa, xb = int(tb["perm"][a]), int(tb["perm"][y])
    frm = np.asarray(gr["frm"])
    to = np.asarray(gr["to"])
    assert modify.find_branch(frm, to, xa, xb) >= 0
    delta = -0.25 * abs(float(G[xa, xb]))
    new = modify.algorithm2(st, frm, to, xa, xb, delta, to_root=True)
    G2 = modify.modified_G(G, xa, xb, delta)
    assert hinv.relative_error(new.dense(), np.linalg.inv(G2)) <= 1e-12


# ---------------------------------------------------------------- three-phase stepping
def _with_loads(net):
    out = dict(net)
    out.update(load_bus=np.array([1, 4, 9], np.int32), load_amp=np.array([0.05, 0.08, 0.03]),
               load_phi=np.array([0.3, -0.2, 1.1]))
    return out


def test_three_phase_stepping_without_mutual_is_three_shifted_single_phase_runs():
    # L_mut = 0 decouples the phases: phase p of every bus follows the single-phase stepping of the
    # same network with its sources and loads shifted by -2 pi p / 3, trip included
    from oracle import emt3
    net = _with_loads(netgen.small_network(13, 77))
    net3 = netgen.three_phase(net)
    net3["L_mut"] = np.zeros(len(net["br_a"]))
    trip = 5
    got, _ = emt3.simulate3(net3, DT, 160, [(80, emt3.TRIP, trip, 0.0)])
    for p in range(3):
        netp = dict(net)
        netp["src_phi"] = np.asarray(net["src_phi"]) + (-2 * np.pi * p / 3)
        netp["load_phi"] = np.asarray(net["load_phi"]) + (-2 * np.pi * p / 3)
        ref, _ = emt.simulate(emt.Network(netp, DT, want_tree=False), 160, [(80, emt.TRIP, trip, 0.0)])
        assert np.max(np.abs(got[:, p::3] - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_three_phase_faults_without_mutual_are_single_phase_faults_on_one_copy():
    # L_mut = 0 decouples the phases: a fault on phase p of a bus acts on the single-phase copy of
    # phase p alone (emt.py's fault semantics, pinned by Kirchhoff balance); the other phases run
    # as if there were no fault. Overlapping windows and a trip inside them included.
    from oracle import emt3
    net = _with_loads(netgen.small_network(13, 77))
    net3 = netgen.three_phase(net)
    net3["L_mut"] = np.zeros(len(net["br_a"]))
    trip = 5
    ev3 = [(40, emt3.FAULT_ON, 3 * 4 + 1, 10.0), (60, emt3.FAULT_ON, 3 * 9 + 1, 5.0), (70, emt3.TRIP, trip, 0.0),
           (90, emt3.FAULT_OFF, 3 * 4 + 1, 0.0), (120, emt3.FAULT_OFF, 3 * 9 + 1, 0.0), (100, emt3.FAULT_ON, 3 * 2 + 2, 20.0)]
    got, state = emt3.simulate3(net3, DT, 160, ev3)
    assert state["faults"] == {13: [], 28: [], 8: [20.0]}
    for p in range(3):
        netp = dict(net)
        netp["src_phi"] = np.asarray(net["src_phi"]) + (-2 * np.pi * p / 3)
        netp["load_phi"] = np.asarray(net["load_phi"]) + (-2 * np.pi * p / 3)
        ev1 = [(70, emt.TRIP, trip, 0.0)]
        for st, kind, x, val in ev3:
            if kind != emt3.TRIP and x % 3 == p:
                ev1.append((st, emt.FAULT_ON if kind == emt3.FAULT_ON else emt.FAULT_OFF, x // 3, val))
        ref, _ = emt.simulate(emt.Network(netp, DT, want_tree=False), 160, ev1)
        assert np.max(np.abs(got[:, p::3] - ref)) <= 1e-12 * np.max(np.abs(ref)), p


def test_three_phase_fault_cleared_where_none_is_on_is_rejected():
    from oracle import emt3
    net = netgen.three_phase(netgen.small_network(13, 77))
    with pytest.raises(ValueError):
        emt3.simulate3(net, DT, 20, [(5, emt3.FAULT_ON, 4, 10.0), (8, emt3.FAULT_OFF, 5, 0.0)])


def test_three_phase_balanced_steady_state_uses_positive_sequence_inductance():
    # Balanced source (Rs) -> coupled RL branch -> bus 1 with a shunt C. Balanced currents sum to
    # zero, so L3 i = (L - L_mut) i per phase; the trapezoidal steady state is the phasor solution
    # with s = j (2/dt) tan(w dt / 2) (bilinear transform), each phase shifted by -2 pi p / 3.
    from oracle import emt3
    f, dt = 60.0, 50e-6
    w = 2 * np.pi * f
    Rs, R, L, M, C0, C1, V, phi = 1.0, 2.0, 10e-3, 3e-3, 20e-6, 100e-6, 1.3, 0.4
    net = dict(n_bus=2, br_a=np.array([0], np.int32), br_b=np.array([1], np.int32), kind=np.array([0], np.int32),
               R=np.array([R]), L=np.array([L]), C=np.zeros(1), L_mut=np.array([M]), shunt_C=np.array([C0, C1]),
               src_bus=np.array([0], np.int32), src_Vm=np.array([V]), src_phi=np.array([phi]),
               src_Rs=np.array([Rs]), load_bus=np.zeros(0, np.int32), load_amp=np.zeros(0), load_phi=np.zeros(0),
               freq=f)
    n = 8000
    out, _ = emt3.simulate3(net, dt, n)
    s = 1j * (2 / dt) * np.tan(w * dt / 2)
    Zb = R + s * (L - M)
    A = np.array([[1 / Rs + s * C0 + 1 / Zb, -1 / Zb], [-1 / Zb, s * C1 + 1 / Zb]])
    k = np.arange(n - 400, n) + 1
    for p in range(3):
        E = V * np.exp(1j * (phi + (-2 * np.pi * p / 3) - np.pi / 2)) / Rs
        Vp = np.linalg.solve(A, np.array([E, 0]))
        ref = np.real(Vp[None, :] * np.exp(1j * w * k * dt)[:, None])
        got = out[n - 400:, [p, 3 + p]]
        assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_three_phase_lossless_network_conserves_energy_exactly():
    # R = 0 and no source resistances: the trapezoidal rule keeps the quadratic invariant
    # 1/2 sum C v^2 + 1/2 sum i^T L3 i (+ series capacitors) once the driving sinks stop
    from oracle import emt3
    net = _with_loads(netgen.small_network(24, 5))
    net.update(src_bus=np.zeros(0, np.int32), src_Vm=np.zeros(0), src_phi=np.zeros(0), src_Rs=np.zeros(0))
    net["R"] = np.zeros(len(net["br_a"]))
    net3 = netgen.three_phase(net)
    kind = np.asarray(net3["kind"])
    assert (kind == cm.KIND_RL).any() and (kind == cm.KIND_RC).any()

    def energy(st):
        v = st["v"]
        E = 0.5 * np.sum(np.repeat(net3["shunt_C"], 3) * v ** 2)
        for e in range(len(kind)):
            i = st["cur"][e]
            if kind[e] == cm.KIND_RL:
                L, M = float(net3["L"][e]), float(net3["L_mut"][e])
                E += 0.5 * i @ ((L - M) * np.eye(3) + M * np.ones((3, 3))) @ i
            else:
                a, b = int(net3["br_a"][e]), int(net3["br_b"][e])
                vc = v[3 * a:3 * a + 3] - v[3 * b:3 * b + 3]   # R = 0: the capacitor holds the branch voltage
                E += 0.5 * float(net3["C"][e]) * vc @ vc
        return E

    # driven by the sinks for 100 steps; then free: the first free step still integrates the sinks at
    # its start, every later one conserves the energy
    _, state = emt3.simulate3(net3, DT, 100, monitor=[0])
    free = dict(net3)
    free.update(load_bus=np.zeros(0, np.int32), load_amp=np.zeros(0), load_phi=np.zeros(0))
    _, state = emt3.simulate3(free, DT, 1, monitor=[0], init=state, first_step=101)
    E0 = energy(state)
    assert E0 > 0
    for k in range(6):
        _, state = emt3.simulate3(free, DT, 50, monitor=[0], init=state, first_step=102 + 50 * k)
        assert abs(energy(state) - E0) <= 1e-11 * E0
