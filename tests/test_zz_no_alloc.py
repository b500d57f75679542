"""emt_apply_noalloc: the single-vector apply for callers that cannot allocate
device memory while they run, such as a real-time simulator loop that reserves
all of its memory at start-up (its scratch is a fixed device array inside the
library). Each case checks the result against the oracle's dense solve and
against emt_apply, on two calls in a row.

Tolerances. FP64 and float-float stores: 1e-10 of the max-norm, as everywhere.
FP32 stores return the unrefined FP32 result; every output element is a sum of
at most m = (largest leaf) + (sum over nodes of 2k) products of stored FP32
values, so by the standard dot-product bound each element is within
m * 2^-24 * (|G^-1| |x|) of the exact solve (componentwise).

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

import netgen
from oracle import emt as oemt
from oracle import hinv as ohinv
from oracle import modify as omod
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = 50e-6
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def L():
    from paper_2105_10661_gb300 import buildlib
    buildlib.build()
    import paper_2105_10661_gb300._lib as lib
    assert torch.cuda.is_available()
    return lib


def _store(L, net, levels, prec, mode=0):
    nw = oemt.Network(net, DT, levels=levels)
    gr = nw.gr
    h = L.emt_build_hinv(gr["n_bus"], gr["frm"], gr["to"], gr["g"], levels=levels, mode=mode, precision=prec)
    return nw, h


def _terms(nw):
    # m of the FP32 bound: the largest leaf plus every node's boundary vector (2k)
    t = nw.tree
    leaves = [p for p in range(len(t["lo"])) if t["left"][p] < 0]
    b = max(int(t["hi"][p] - t["lo"][p]) for p in leaves)
    return b + 2 * int(t["cut_ptr"][-1])


def _calls(L, h, n, seed, G, prec, m):
    # two calls in a row; each result against the dense solve of G and against emt_apply
    rng = np.random.default_rng(seed)
    Ginv = np.linalg.inv(G)
    for call in range(2):
        x = rng.standard_normal(n)
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        v_new = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        v_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        L.emt_apply_noalloc(h, xd, v_new)
        L.emt_apply(h, xd, v_ref)
        torch.cuda.synchronize()
        got, api = v_new.cpu().numpy(), v_ref.cpu().numpy()
        exact = Ginv @ x
        assert np.all(np.isfinite(got)), call
        if prec == 2:
            bound = m * U32 * (np.abs(Ginv) @ np.abs(x))
            assert np.all(np.abs(got - exact) <= bound), (call, float(np.max(np.abs(got - exact) / bound)))
            assert np.all(np.abs(got - api) <= 2 * bound), call
        else:
            assert rel_err(got, exact) <= 1e-10, (call, rel_err(got, exact))
            assert rel_err(got, api) <= 1e-10, (call, rel_err(got, api))


@pytest.mark.parametrize("prec", [1, 0, 2])
def test_noalloc_first_call_on_a_fresh_store_matches_the_dense_solve(L, prec):
    # the very first apply on the store is the no-allocation one (nothing prepared by emt_apply)
    net = netgen.tiled(2, 4)
    nw, h = _store(L, net, 3, prec)
    _calls(L, h, net["n_bus"], 21, nw.G, prec, _terms(nw))


@pytest.mark.parametrize("prec", [1, 2])
def test_noalloc_after_a_trip_and_a_fault_matches_the_dense_solve(L, prec):
    # the modification rewrites the store's blocks, cut conductances and packed copies; the
    # no-allocation apply reads them directly
    net = netgen.tiled(2, 4)
    nw, h = _store(L, net, 3, prec)
    x = torch.ones(net["n_bus"], dtype=torch.float64, device="cuda")
    v = torch.zeros_like(x)
    L.emt_apply_noalloc(h, x, v)
    e = netgen.pick_branch(net)
    a, b, g = int(nw.series_frm[e]), int(nw.series_to[e]), float(nw.g_series[e])
    L.emt_modify_branch(h, a, b, -g)
    G = omod.modified_G(nw.G, a, b, -g)
    _calls(L, h, net["n_bus"], 23, G, prec, _terms(nw))
    L.emt_modify_branch(h, 700, -1, 0.1)
    G = omod.modified_G(G, 700, -1, 0.1)
    _calls(L, h, net["n_bus"], 24, G, prec, _terms(nw))


def test_noalloc_paper_store_matches_algorithm1(L):
    net = netgen.tile(1_000_000)
    nw, h = _store(L, net, 2, 1, mode=1)
    H = ohinv.HInv(nw.G, nw.tree, nw.g_series, ohinv.PAPER)
    rng = np.random.default_rng(25)
    for call in range(2):
        x = rng.standard_normal(net["n_bus"])
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        v_new = torch.full_like(xd, np.nan)
        v_ref = torch.zeros_like(xd)
        L.emt_apply_noalloc(h, xd, v_new)
        L.emt_apply(h, xd, v_ref)
        torch.cuda.synchronize()
        got = v_new.cpu().numpy()
        assert rel_err(got, H.apply(x)) <= 1e-10, call
        assert rel_err(got, v_ref.cpu().numpy()) <= 1e-10, call


def test_noalloc_small_ragged_store(L):
    net = netgen.small_network(37, 5)
    nw, h = _store(L, net, 3, 1)
    _calls(L, h, 37, 22, nw.G, 1, _terms(nw))


def test_noalloc_rejects_a_store_beyond_its_fixed_scratch(L):
    # 9 x 8 tiles in 8 leaves of about 1,611 buses need 8 * 51 * 1,612 * 8 bytes (5.3 MB) of
    # partial sums, more than the 4 MiB array: rejected before any launch, emt_apply still works
    net = netgen.tiled(9, 8)
    gr = oemt.Network(net, DT, want_tree=False).gr
    h = L.emt_build_hinv(gr["n_bus"], gr["frm"], gr["to"], gr["g"], levels=3, precision=1)
    n = net["n_bus"]
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    v = torch.full_like(x, -7.0)
    with pytest.raises(L.EmtError) as ex:
        L.emt_apply_noalloc(h, x, v)
    assert ex.value.code == L.EMT_ERR_UNSUPPORTED
    assert "EMT_APPLY_NOALLOC_SCRATCH_BYTES" in str(ex.value)
    torch.cuda.synchronize()
    assert torch.all(v == -7.0)
    L.emt_apply(h, x, v)
    torch.cuda.synchronize()
    assert torch.isfinite(v).all()


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("levels,d_th", [(3, 0), (0, 12)])
def test_noalloc_on_a_random_multigraph_store_matches_the_dense_solve(L, prec, levels, d_th):
    # an irregular tree (hub cuts, parallel branches, isolated buses with only a shunt), then a
    # trip of one branch of a parallel pair
    n, a, b = netgen.random_multigraph(41)
    rng = np.random.default_rng(141)
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
    h = L.emt_build_hinv(n, frm, to, gv, levels=levels, d_th=d_th, precision=prec)
    _calls(L, h, n, 1, G, prec, 0)
    L.emt_modify_branch(h, int(frm[0]), int(to[0]), -float(gv[0]))
    u = np.zeros(n)
    u[frm[0]] = 1.0
    u[to[0]] = -1.0
    _calls(L, h, n, 2, G - gv[0] * np.outer(u, u), prec, 0)
