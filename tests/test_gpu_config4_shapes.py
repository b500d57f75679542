"""GPU parity at the full shapes of the 11,456-bus, 512-scenario workload.

The multi-column simulation runs the whole 11,456-bus network (64 tiles with
loads, 4-level hierarchy: 16 leaves of 716 buses, so 6 row tiles and 23 K
chunks of the tensor-core leaf product per leaf) with all 512 scenario columns
(three 192-column tiles, the last one ragged). Eight columns (first, last, both
sides of the tile edge at 192, the middle and the ragged tile) are compared
element by element with the CPU oracle (FP64, exact hierarchical store) over
every step: the monitored buses at every step and every bus at the last step.
Tolerance 1e-8 of the max-norm (split-BF16 products refined once per step
against the float-float residual)."""
import numpy as np
import pytest

import netgen
from oracle import emt as oemt
from tests.gpu_util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = 50e-6
R = 512
STEPS = 12
COLS = [0, 1, 191, 192, 256, 447, 510, 511]


@pytest.fixture(scope="module")
def L():
    from paper_2105_10661_gb300 import buildlib
    buildlib.build()
    import paper_2105_10661_gb300._lib as lib
    assert torch.cuda.is_available()
    return lib


@pytest.fixture(scope="module")
def case():
    net = netgen.config_network(4)
    ss, ls = netgen.scenario_scales(net, R, seed=13)
    mon = np.sort(np.random.default_rng(17).choice(net["n_bus"], 256, replace=False))
    nw = oemt.Network(net, DT, levels=4)
    refs = {}
    for c in COLS:
        traj, state = oemt.simulate(nw, STEPS, [], solver="exact", src_scale=ss[c], load_scale=ls[c])
        refs[c] = (traj[:, mon], state["v"])
    return net, ss, ls, mon, refs


@pytest.mark.parametrize("kernels", [None, 3])
def test_scenarios_11456_buses_512_columns_match_oracle(L, case, kernels):
    # kernels None: the products emt_sim_create picks (tensor-core leaf GEMM, 192-column tiles);
    # 3: tensor cores for the expansion as well
    net, ss, ls, mon, refs = case
    n = net["n_bus"]
    sim = L.emt_sim_create(net, DT, levels=4, nrhs=R, src_scale=ss, load_scale=ls)
    if kernels is not None:
        L.emt_sim_tune(sim, 0, kernels)
    L.emt_sim_monitor(sim, mon)
    rec = torch.zeros(STEPS, R, len(mon), dtype=torch.float64, device="cuda")
    h1 = STEPS // 2
    L.emt_step(sim, h1, rec[:h1])
    L.emt_step(sim, STEPS - h1, rec[h1:])
    torch.cuda.synchronize()
    got = rec.cpu().numpy()
    final = L.emt_sim_read(sim, 0).reshape(R, n)
    assert np.all(np.isfinite(got))
    for c in COLS:
        traj, v_last = refs[c]
        assert rel_err(got[:, c, :], traj) <= 1e-8, (c, rel_err(got[:, c, :], traj))
        assert rel_err(final[c], v_last) <= 1e-8, (c, rel_err(final[c], v_last))
