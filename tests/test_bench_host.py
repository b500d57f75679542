"""Host logic of the benchmark (no GPU): the clock record taken during the timed
region, and the whole-job rate of independent replicas."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _row(sm, mx, hw="Not Active", hw_th="Not Active", sw_th="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 812.35, 0x0000000000000000, {hw}, {hw_th}, {sw_th}, {cap}\n"


def test_clock_summary_median_max_and_reasons():
    lines = [_row(2070, 2070), _row(1995, 2070, cap="Active"), _row(2040, 2070), "garbage\n",
             _row("[N/A]", 2070)]
    c = bench.summarize_clocks(lines)
    assert c["samples"] == 4
    assert c["sm_mhz"] == pytest.approx(2040.0)     # median of 2070, 1995, 2040
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_every_throttle_kind():
    lines = [_row(1400, 2070, hw="Active"), _row(1400, 2070, hw_th="Active"), _row(1400, 2070, sw_th="Active")]
    assert bench.summarize_clocks(lines)["reasons"] == ["hw_slowdown", "hw_thermal_slowdown",
                                                        "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    c = bench.summarize_clocks([])
    assert c == {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}


def test_job_rate_counts_every_rank():
    # 4 replicas, 1,432 buses x 20,000 steps each, slowest rank 100 ms
    assert bench.job_rate(1432 * 20000, 4, 100.0) == pytest.approx(4 * 1432 * 20000 / 0.1)


# ---- solve FLOP counts of Sec. V-B (hierarchical store against sparse LU)

def test_lu_flops_closed_forms():
    # path graph: tridiagonal, no fill; the Thomas algorithm's 3(n - 1) and 5n - 4
    n = 50
    c = bench.lu_flops(n, list(range(n - 1)), list(range(1, n)))
    assert (c["factor"], c["solve"]) == (3 * (n - 1), 5 * n - 4)
    # complete graph: dense LU, sum over pivots of j divisions and j^2 multiply-adds
    m = 9
    a, b = zip(*[(i, j) for i in range(m) for j in range(i + 1, m)])
    c = bench.lu_flops(m, a, b)
    assert c["factor"] == sum(j + 2 * j * j for j in range(m))
    assert c["solve"] == 2 * m * m - m


def _counting_apply(H, p, x, ops, paper):
    """The solve of the store of node p's subtree, node by node in the recursive order of Eq. 9
    with the cut-row gather t_p = [h_l^T y_l; h_r^T y_r], counting every addition and
    multiplication. PAPER cores [[0, I], [I, 0]] are applied as the swap they are."""
    t = H.tree
    if t["left"][p] < 0:
        Lj = H.leaf_inv[p]
        y = []
        for i in range(len(x)):
            acc = Lj[i, 0] * x[0]
            ops[0] += 1
            for j in range(1, len(x)):
                acc += Lj[i, j] * x[j]
                ops[0] += 2
            y.append(acc)
        return y
    l, r = int(t["left"][p]), int(t["right"][p])
    nl = int(t["hi"][l] - t["lo"][l])
    yl = _counting_apply(H, l, x[:nl], ops, paper)
    yr = _counting_apply(H, r, x[nl:], ops, paper)
    hl, hr, P, Q, C = H.hl[p], H.hr[p], H.P[p], H.Q[p], H.C[p]
    k = P.shape[1]
    if k == 0:
        return yl + yr
    tv = []
    for e in range(k):   # h_l column e = -g_e at row a_e: one product
        a = int(np.nonzero(hl[:, e])[0][0])
        tv.append(hl[a, e] * yl[a])
        ops[0] += 1
    for e in range(k):   # h_r column e = unit vector at row b_e: a gather
        tv.append(yr[int(np.nonzero(hr[:, e])[0][0])])
    if paper:
        s = tv[k:] + tv[:k]
    else:
        s = []
        for i in range(2 * k):
            acc = C[i, 0] * tv[0]
            ops[0] += 1
            for j in range(1, 2 * k):
                acc += C[i, j] * tv[j]
                ops[0] += 2
            s.append(acc)
    out = []
    for F, y, half in ((P, yl, s[:k]), (Q, yr, s[k:])):
        for i in range(len(y)):
            acc = F[i, 0] * half[0]
            ops[0] += 1
            for j in range(1, k):
                acc += F[i, j] * half[j]
                ops[0] += 2
            out.append(y[i] - acc)
            ops[0] += 1
    return out


def _counting_leaf_inverse(A, ops):
    """Cholesky A = L L^T, W = L^-1, then A^-1 = W^T W (one triangle, mirrored), counting every
    addition, multiplication, division and square root."""
    b = A.shape[0]
    Lc = np.zeros((b, b))
    for j in range(b):
        acc = A[j, j]
        for k in range(j):
            acc -= Lc[j, k] * Lc[j, k]
            ops[0] += 2
        Lc[j, j] = acc ** 0.5
        ops[0] += 1
        for i in range(j + 1, b):
            acc = A[i, j]
            for k in range(j):
                acc -= Lc[i, k] * Lc[j, k]
                ops[0] += 2
            Lc[i, j] = acc / Lc[j, j]
            ops[0] += 1
    W = np.zeros((b, b))
    for j in range(b):
        W[j, j] = 1.0 / Lc[j, j]
        ops[0] += 1
        for i in range(j + 1, b):
            acc = Lc[i, j] * W[j, j]
            ops[0] += 1
            for k in range(j + 1, i):
                acc += Lc[i, k] * W[k, j]
                ops[0] += 2
            W[i, j] = -acc / Lc[i, i]
            ops[0] += 1
    out = np.zeros((b, b))
    for j in range(b):
        for i in range(j + 1):
            acc = W[j, i] * W[j, j]
            ops[0] += 1
            for k in range(j + 1, b):
                acc += W[k, i] * W[k, j]
                ops[0] += 2
            out[i, j] = out[j, i] = acc
    return out


def _network(n_bus, levels, mode):
    import netgen
    from oracle import emt as oemt
    from oracle import hinv as ohinv
    nw = oemt.Network(netgen.small_network(n_bus, 77), 50e-6, levels=levels)
    return nw, ohinv.HInv(nw.G, nw.tree, nw.g_series, mode)


@pytest.mark.parametrize("paper", [False, True])
@pytest.mark.parametrize("n_bus,levels", [(13, 2), (37, 3)])
def test_hier_solve_flops_counts_a_real_solve(n_bus, levels, paper):
    from oracle import hinv as ohinv
    nw, H = _network(n_bus, levels, ohinv.PAPER if paper else ohinv.EXACT)
    x = np.random.default_rng(4).standard_normal(n_bus)
    ops = [0]
    perm = nw.tree["perm"]
    y = np.array(_counting_apply(H, 0, list(x[perm]), ops, paper))
    ref = H.apply(x)[perm] if paper else np.linalg.solve(nw.G, x)[perm]   # Algorithm 1's inverse, or exact
    assert np.allclose(y, ref, rtol=1e-10, atol=1e-12)   # the counted loop is the solve
    assert ops[0] == bench.hier_solve_flops(nw.tree, paper=paper)


@pytest.mark.parametrize("n_bus,levels", [(13, 2), (37, 3)])
def test_alg1_build_flops_counts_a_real_build(n_bus, levels):
    """Algorithm 1 with counted loops: direct leaf inverses, then every cut column of P and Q as a
    counted solve through the child's store; each block equals the oracle's PAPER store."""
    from oracle import hinv as ohinv
    nw, H = _network(n_bus, levels, ohinv.PAPER)
    t = nw.tree
    ops = [0]
    for p in range(len(t["lo"])):
        lo, hi = int(t["lo"][p]), int(t["hi"][p])
        if t["left"][p] < 0:
            inv = _counting_leaf_inverse(H.Gp[lo:hi, lo:hi], ops)
            assert np.allclose(inv, H.leaf_inv[p], rtol=1e-10, atol=1e-13)
            continue
        for child, h, F in ((int(t["left"][p]), H.hl[p], H.P[p]), (int(t["right"][p]), H.hr[p], H.Q[p])):
            for e in range(h.shape[1]):
                col = np.array(_counting_apply(H, child, list(h[:, e]), ops, True))
                assert np.allclose(col, F[:, e], rtol=1e-10, atol=1e-13)
    assert ops[0] == bench.alg1_build_flops(t)


@pytest.mark.parametrize("to_ground", [False, True])
def test_alg2_flops_counts_a_real_modification(to_ground):
    """Algorithm 2 with counted loops on the touched leaves and path nodes (the oracle's own path
    logic picks them): a trip of a root cut branch, or a fault to ground; the recomputed blocks
    equal the oracle's Algorithm 2."""
    from oracle import hinv as ohinv
    from oracle import modify as omod
    nw, H = _network(37, 3, ohinv.PAPER)
    t = nw.tree
    c0 = int(t["cut_ptr"][0])
    a, b = int(t["cut_a"][c0]), int(t["cut_b"][c0])
    if to_ground:
        b, delta = -1, 0.1
    else:
        delta = -float(nw.g_series[int(t["cut_e"][c0])])
    perm = t["perm"]
    new = omod.algorithm2(H, nw.series_frm, nw.series_to, int(perm[a]), int(perm[b]) if b >= 0 else -1, delta)
    leaves, order, _ = omod.touched_path(t, a, b, False)
    ops = [0]
    for j in leaves:
        lo, hi = int(t["lo"][j]), int(t["hi"][j])
        assert np.allclose(_counting_leaf_inverse(new.Gp[lo:hi, lo:hi], ops), new.leaf_inv[j], rtol=1e-10,
                           atol=1e-13)
    for q in order:
        for child, h, F in ((int(t["left"][q]), new.hl[q], new.P[q]), (int(t["right"][q]), new.hr[q], new.Q[q])):
            for e in range(h.shape[1]):
                col = np.array(_counting_apply(new, child, list(h[:, e]), ops, True))
                assert np.allclose(col, F[:, e], rtol=1e-10, atol=1e-13)
    assert ops[0] == bench.alg2_flops(t, a, b)
    assert (len(order) == 0) == to_ground


def test_hier_solve_flops_single_leaf_is_dense_matvec():
    n = 20
    tree = {"lo": [0], "hi": [n], "left": [-1], "right": [-1], "cut_ptr": [0, 0]}
    assert bench.hier_solve_flops(tree) == 2 * n * n - n
    assert bench.leaf_inverse_flops(1) == 3   # sqrt, reciprocal, one product


def test_flop_table_row_on_one_tile():
    rows = bench.flop_table(shapes=((1, 1),), dths=(45, 179))
    r = rows[0]
    assert r["n_bus"] == 179
    assert r["solve_paper_dth179"] == r["dense_matvec"] == 2 * 179 * 179 - 179   # one leaf: the dense inverse
    assert r["alg1_build_dth179"] == bench.leaf_inverse_flops(179)
    assert r["alg2_fault_dth179"] == r["alg1_build_dth179"]                       # the only leaf is touched
    assert "alg2_root_trip_dth179" not in r                                       # a single leaf has no cuts
    assert r["solve_paper_dth45"] < r["solve_exact_dth45"] < r["dense_matvec"]
    assert r["alg2_fault_dth45"] < r["alg2_root_trip_dth45"] < r["alg1_build_dth45"]
