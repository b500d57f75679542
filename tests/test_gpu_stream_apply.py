"""GPU parity of the streaming apply: stores whose leaf blocks exceed the caches (the
11,456-bus network, 16 leaves of 716 buses, 64 MB of leaf blocks) are applied by the
HBM streaming kernels. Reference: the exact solve of G v = i by sparse LU (SciPy), before
and after local modifications of the store (line trips), to 1e-10."""
import numpy as np
import pytest

import netgen
from oracle import companion as ocomp
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
spla = pytest.importorskip("scipy.sparse.linalg")
pytestmark = pytest.mark.gpu

DT = 50e-6


@pytest.fixture(scope="module")
def L():
    from paper_2105_10661_gb300 import buildlib
    buildlib.build()
    import paper_2105_10661_gb300._lib as lib
    assert torch.cuda.is_available()
    return lib


@pytest.fixture(scope="module")
def big():
    net = netgen.config_network(4)
    gr = ocomp.graph(net, DT)
    return net, gr


def _apply(L, h, X, pos_in=False):
    n, m = X.shape
    i_dev = torch.tensor(X.T.copy(), dtype=torch.float64, device="cuda")
    v_dev = torch.zeros_like(i_dev)
    L.emt_apply(h, i_dev, v_dev, nrhs=m, ld=n)
    torch.cuda.synchronize()
    return v_dev.cpu().numpy().T


@pytest.mark.parametrize("mode", [2, 0])
@pytest.mark.parametrize("prec", [0, 1])
def test_streaming_apply_matches_sparse_solve_and_tracks_trips(L, big, prec, mode):
    # mode 2: the single cooperative launch; 0: the default, three chained kernels
    net, gr = big
    n = net["n_bus"]
    G = ocomp.assemble_sparse(gr).tocsc()
    h = L.emt_build_hinv_from_network(net, DT, levels=4, precision=prec)
    L.emt_apply_tune(h, mode)
    X = np.random.default_rng(21).standard_normal((n, 3))
    assert rel_err(_apply(L, h, X), spla.splu(G).solve(X)) <= 1e-10
    assert L.emt_apply_tune(h, mode) == (2 if mode == 2 else 1)
    # two trips: one branch inside a leaf, one chosen by the seeded picker (may cross leaves)
    rng = np.random.default_rng(5)
    for e in [netgen.pick_branch(net), int(rng.integers(0, gr["n_series"]))]:
        a, b, g = int(gr["frm"][e]), int(gr["to"][e]), float(gr["g"][e])
        L.emt_modify_branch(h, a, b, -g)
        G = G.tolil()
        G[a, a] -= g
        G[b, b] -= g
        G[a, b] += g
        G[b, a] += g
        G = G.tocsc()
        assert rel_err(_apply(L, h, X), spla.splu(G).solve(X)) <= 1e-10


def test_streaming_apply_repeatable_bit_for_bit(L, big):
    net, _ = big
    n = net["n_bus"]
    h = L.emt_build_hinv_from_network(net, DT, levels=4, precision=1)
    X = np.random.default_rng(3).standard_normal((n, 1))
    a = _apply(L, h, X)
    b = _apply(L, h, X)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", [0, 1])
def test_single_launch_apply_repeats_bit_for_bit_and_agrees_with_three_kernels(L, big, prec):
    # many launches in a row: the grid-barrier counters return to zero after every launch
    net, _ = big
    n = net["n_bus"]
    h = L.emt_build_hinv_from_network(net, DT, levels=4, precision=prec)
    x = torch.tensor(np.random.default_rng(8).standard_normal(n), dtype=torch.float64, device="cuda")
    first = torch.zeros_like(x)
    L.emt_apply_tune(h, 2)
    L.emt_apply(h, x, first)
    assert L.emt_apply_tune(h, 2) == 2
    outs = [torch.zeros_like(x) for _ in range(40)]
    for o in outs:
        L.emt_apply(h, x, o)
    L.emt_hinv_sync(h)
    for o in outs:
        assert torch.equal(o, first)
    L.emt_apply_tune(h, 1)
    three = torch.zeros_like(x)
    L.emt_apply(h, x, three)
    torch.cuda.synchronize()
    assert rel_err(first.cpu().numpy(), three.cpu().numpy()) <= 1e-13


@pytest.mark.parametrize("warps", [4, 7, 12, 16])
def test_single_launch_warp_counts_match_sparse_solve(L, big, warps):
    # 4..16 warps per CTA, each streaming its own rows (ragged last rounds in every CTA)
    net, gr = big
    n = net["n_bus"]
    G = ocomp.assemble_sparse(gr).tocsc()
    h = L.emt_build_hinv_from_network(net, DT, levels=4, precision=1)
    L.emt_apply_tune(h, 2, warps)
    X = np.random.default_rng(31).standard_normal((n, 2))
    got = _apply(L, h, X)
    assert L.emt_apply_tune(h, 2, warps) == 2
    assert rel_err(got, spla.splu(G).solve(X)) <= 1e-10
