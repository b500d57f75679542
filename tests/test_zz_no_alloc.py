"""emt_apply_noalloc: the single-vector apply for callers that cannot allocate
device memory while running (its scratch is a fixed device array inside the
library). It must give the same answer as emt_apply, call after call.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
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


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-10), (2, 1e-6)])
def test_noalloc_matches_emt_apply_two_calls(L, prec, tol):
    net = netgen.tiled(2, 4)
    gr = oemt.Network(net, DT, want_tree=False).gr
    h = L.emt_build_hinv(gr["n_bus"], gr["frm"], gr["to"], gr["g"], levels=3, mode=L.EMT_MODE_EXACT, precision=prec)
    n = net["n_bus"]
    rng = np.random.default_rng(21)
    for call in range(2):
        x = torch.tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda")
        v_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        v_new = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        L.emt_apply(h, x, v_ref)
        L.emt_apply_noalloc(h, x, v_new)
        torch.cuda.synchronize()
        got, ref = v_new.cpu().numpy(), v_ref.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert rel_err(got, ref) <= tol, (call, rel_err(got, ref))


def test_noalloc_small_ragged_store(L):
    net = netgen.small_network(37, 5)
    gr = oemt.Network(net, DT, want_tree=False).gr
    h = L.emt_build_hinv(gr["n_bus"], gr["frm"], gr["to"], gr["g"], levels=3, precision=L.EMT_PREC_FF64)
    rng = np.random.default_rng(22)
    for call in range(2):
        x = torch.tensor(rng.standard_normal(37), dtype=torch.float64, device="cuda")
        v_ref = torch.zeros(37, dtype=torch.float64, device="cuda")
        v_new = torch.zeros(37, dtype=torch.float64, device="cuda")
        L.emt_apply(h, x, v_ref)
        L.emt_apply_noalloc(h, x, v_new)
        torch.cuda.synchronize()
        assert rel_err(v_new.cpu().numpy(), v_ref.cpu().numpy()) <= 1e-10
