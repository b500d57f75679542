"""Host-side checks of the native library (no GPU): it loads, exports every
entry point of include/emt.h, and its partition tree is bit-exact with the
oracle's independent implementation."""
import os
import re

import numpy as np
import pytest

import netgen
from oracle import partition as opart

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2105_10661_gb300 import buildlib
    buildlib.build()
    import paper_2105_10661_gb300._lib as lib
    return lib


def test_exports_every_declared_symbol(L):
    hdr = open(os.path.join(ROOT, "include", "emt.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"\b(emt_[a-z_0-9]+)\s*\(", hdr))
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(L.lib, name), name
    assert set(L.EXPORTED) == declared


KEYS = ["perm", "lo", "hi", "parent", "left", "right", "depth", "cut_ptr", "cut_a", "cut_b", "cut_e"]


@pytest.mark.parametrize("which,levels,d_th", [
    ("tile", 2, 0), ("tile", 0, 74), ("tile", 0, 10), ("tile", 0, 2), ("tiles8", 3, 0), ("tiles8", 0, 100),
    ("small5", 2, 0), ("small13", 3, 0), ("small37", 0, 7), ("small2", 1, 0)])
def test_partition_bit_exact_with_oracle(L, which, levels, d_th):
    if which == "tile":
        net = netgen.tile(1_000_000)
    elif which == "tiles8":
        net = netgen.tiled(2, 4)
    else:
        net = netgen.small_network(int(which[5:]), 77)
    got = L.emt_tree_build(net["n_bus"], net["br_a"], net["br_b"], levels=levels, d_th=d_th)
    ref = opart.build_tree(net["n_bus"], net["br_a"], net["br_b"], levels=levels, d_th=d_th)
    for k in KEYS:
        assert np.array_equal(got[k], np.asarray(ref[k])), k


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("levels,d_th", [(3, 0), (0, 9)])
def test_partition_bit_exact_on_random_multigraphs(L, seed, levels, d_th):
    n, a, b = netgen.random_multigraph(seed)
    got = L.emt_tree_build(n, a, b, levels=levels, d_th=d_th)
    ref = opart.build_tree(n, a, b, levels=levels, d_th=d_th)
    for k in KEYS:
        assert np.array_equal(got[k], np.asarray(ref[k])), k


def test_partition_bit_exact_64_tiles(L):
    net = netgen.config_network(4)
    got = L.emt_tree_build(net["n_bus"], net["br_a"], net["br_b"], levels=4)
    ref = opart.build_tree(net["n_bus"], net["br_a"], net["br_b"], levels=4)
    for k in KEYS:
        assert np.array_equal(got[k], np.asarray(ref[k])), k


@pytest.mark.parametrize("which,levels,d_th", [("tile", 2, 0), ("tiles8", 3, 0), ("small40", 0, 24), ("tiles8", 0, 300)])
def test_block_partition_bit_exact_with_oracle(L, which, levels, d_th):
    # three nodes per bus: the partition bisects buses and cuts in rank-3 blocks
    from oracle import companion as ocm
    base = (netgen.tile(1_000_000) if which == "tile" else netgen.tiled(2, 4) if which == "tiles8"
            else netgen.small_network(int(which[5:]), 77))
    gr = ocm.three_phase_graph(netgen.three_phase(base), 50e-6)
    got = L.emt_tree_build(gr["n_bus"], gr["frm"], gr["to"], levels=levels, d_th=d_th, nodes_per_bus=3)
    ref = opart.build_block_tree(gr["n_bus"], gr["frm"], gr["to"], 3, levels=levels, d_th=d_th)
    for k in KEYS:
        if k == "cut_a":
            a = np.asarray(ref["cut_a"]).reshape(-1, 3)
            assert np.array_equal(a - a[:, :1], np.tile(np.arange(3), (len(a), 1)))
            assert np.array_equal(got["cut_a"], a[:, 0])
        else:
            assert np.array_equal(got[k], np.asarray(ref[k])), k
    assert len(got["cut_b"]) > 0


@pytest.mark.parametrize("seed", [11, 12, 13])
@pytest.mark.parametrize("levels,d_th", [(2, 0), (0, 8)])
def test_block_partition_bit_exact_on_random_multigraphs(L, seed, levels, d_th):
    # vertices grouped in threes: the random multigraph's buses become groups, and each of its
    # branches joins a random vertex of one group to a random vertex of the other
    n, a, b = netgen.random_multigraph(seed)
    rng = np.random.default_rng(seed)
    fa = 3 * a + rng.integers(0, 3, len(a))
    fb = 3 * b + rng.integers(0, 3, len(b))
    got = L.emt_tree_build(3 * n, fa, fb, levels=levels, d_th=d_th, nodes_per_bus=3)
    ref = opart.build_block_tree(3 * n, fa, fb, 3, levels=levels, d_th=d_th)
    for k in KEYS:
        if k == "cut_a":
            assert np.array_equal(got["cut_a"], np.asarray(ref["cut_a"]).reshape(-1, 3)[:, 0])
        else:
            assert np.array_equal(got[k], np.asarray(ref[k])), k


def test_block_partition_rejects_a_vertex_count_off_the_group_size(L):
    with pytest.raises(L.EmtError) as e:
        L.emt_tree_build(7, [0, 3], [3, 6], levels=1, nodes_per_bus=3)
    assert e.value.code == L.EMT_ERR_INVALID


def test_partition_rejects_bad_input(L):
    with pytest.raises(L.EmtError) as e:
        L.emt_tree_build(4, [0, 1], [1, 7], levels=1)
    assert e.value.code == L.EMT_ERR_INVALID
    with pytest.raises(L.EmtError):
        L.emt_tree_build(4, [0], [1], levels=0, d_th=0)


def test_partition_accessor_rejects_null_handle(L):
    assert L.lib.emt_hinv_get_partition(None, None, None, None, None) == L.EMT_ERR_INVALID
    assert "null handle" in L.lib.emt_last_error().decode()


def test_network_input_checks_run_before_any_device_work(L):
    # bad element data is rejected on the host with EMT_ERR_INVALID (no GPU needed to see it)
    import ctypes as C
    net = netgen.small_network(5, 3)
    nw, keep = L.make_network(net)
    opts = L.make_opts(levels=1)

    def build(n):
        h = C.c_void_p()
        return L.lib.emt_build_hinv_from_network(C.byref(n), 50e-6, C.byref(opts), None, C.byref(h))

    bad = L.EmtNetwork.from_buffer_copy(nw)
    bad.from_ = None
    assert build(bad) == L.EMT_ERR_INVALID and b"null branch arrays" in L.lib.emt_last_error()
    bad = L.EmtNetwork.from_buffer_copy(nw)
    bad.n_bus = 0
    assert build(bad) == L.EMT_ERR_INVALID and b"sizes" in L.lib.emt_last_error()
    bad = L.EmtNetwork.from_buffer_copy(nw)
    bad.src_Rs = None
    assert build(bad) == L.EMT_ERR_INVALID and b"source" in L.lib.emt_last_error()
    bad = L.EmtNetwork.from_buffer_copy(nw)
    bad.L = None
    assert build(bad) == L.EMT_ERR_INVALID and b"null L" in L.lib.emt_last_error()
    h = C.c_void_p()
    assert L.lib.emt_build_hinv_from_network(C.byref(nw), -1.0, C.byref(opts), None, C.byref(h)) == L.EMT_ERR_INVALID


@pytest.mark.parametrize("frm,to,g,mode,msg", [
    ([0, 1, 2], [1, 2, 7], [1.0, 1.0, 1.0], 0, b"out of range"),
    ([0, 1, 2], [1, 2, 3], [1.0, 0.0, 1.0], 0, b"nonzero"),
    ([0, 1, 2], [1, 1, 3], [1.0, 1.0, 1.0], 0, b"self-loop"),
    ([0, 1, 2], [1, 2, 3], [1.0, 1.0, 1.0], 5, b"bad mode")])
def test_graph_input_checks_run_before_any_device_work(L, frm, to, g, mode, msg):
    import ctypes as C
    gr, keep = L.make_graph(4, frm, to, g)
    o = L.make_opts(levels=1, mode=mode)
    h = C.c_void_p()
    assert L.lib.emt_build_hinv(C.byref(gr), C.byref(o), None, C.byref(h)) == L.EMT_ERR_INVALID
    assert msg in L.lib.emt_last_error()
    assert h.value is None


@pytest.mark.parametrize("field,msg", [("from_", b"null branch arrays"), ("R", b"null branch arrays"),
                                       ("src_Vm", b"null source arrays"), ("load_bus", b"null load arrays")])
@pytest.mark.parametrize("nrhs", [1, 8])
def test_simulation_input_checks_run_before_any_device_work(L, field, msg, nrhs):
    # single- and multi-column simulations reject incomplete element data with a status, not a crash
    import ctypes as C
    nw, keep = L.make_network(netgen.small_network(5, 3))
    bad = L.EmtNetwork.from_buffer_copy(nw)
    setattr(bad, field, None)
    if field == "load_bus":
        bad.n_load = 2
    opts = L.make_opts(levels=1)
    h = C.c_void_p()
    assert L.lib.emt_sim_create(C.byref(bad), C.byref(opts), 50e-6, nrhs, None, None, None,
                                C.byref(h)) == L.EMT_ERR_INVALID
    assert msg in L.lib.emt_last_error()
    assert L.lib.emt_sim_create(None, C.byref(opts), 50e-6, nrhs, None, None, None, C.byref(h)) == L.EMT_ERR_INVALID


def test_server_create_checks_its_arguments(L):
    import ctypes as C
    s = C.c_void_p()
    assert L.lib.emt_server_create(0, 0, C.byref(s)) == L.EMT_ERR_INVALID
    assert b"tick" in L.lib.emt_last_error()


NULL_HANDLE_CALLS = {
    "emt_tree_sizes": (None, None, None, None),
    "emt_tree_arrays": (None,) * 12,
    "emt_hinv_get_partition": (None,) * 5,
    "emt_apply": (None, None, None, 1, 1, 0, 0.0, None),
    "emt_apply_noalloc": (None, None, None, None),
    "emt_modify_branch": (None, 0, 1, -1.0, None),
    "emt_hinv_sync": (None, None),
    "emt_apply_tune": (None, 0, 0, None),
    "emt_sim_schedule": (None, 1, 0, 0, 0.0, -1),
    "emt_sim_monitor": (None, 0, None),
    "emt_step": (None, 1, None, None),
    "emt_sim_read": (None, 0, None),
    "emt_sim_set_rows_per_cta": (None, 0),
    "emt_sim_tune": (None, 0, 2),
    "emt_sim_autotune": (None, 1, None, None, None),
    "emt_sim_set_inject": (None, 0, 0),
    "emt_sim_reset": (None, None),
    "emt_sim_stats": (None, None, 0),
    "emt_sim_bench_kernel": (None, 0, 1, None),
    "emt_server_add_network": (None, None, None, 50e-6, 4, 1, None, None),
    "emt_server_submit": (None, 0, 0.0, 1, -1, 0, 0.0, 0, 0, None),
    "emt_server_submit_network": (None, None, None, 50e-6, 1, None, 0.0, 1, -1, 0, 0.0, 0, 0, None),
    "emt_server_run": (None,),
    "emt_server_result": (None, 0, None, None),
    "emt_server_stats": (None, None, 0),
}


@pytest.mark.parametrize("name", sorted(NULL_HANDLE_CALLS))
def test_every_call_rejects_a_null_handle_with_a_status(L, name):
    # the ABI never throws or aborts: a null handle is EMT_ERR_INVALID with a message
    assert getattr(L.lib, name)(*NULL_HANDLE_CALLS[name]) == L.EMT_ERR_INVALID
    assert L.lib.emt_last_error()


def test_destroy_and_accessors_accept_null(L):
    for name in ("emt_tree_destroy", "emt_hinv_destroy", "emt_sim_destroy", "emt_server_destroy"):
        getattr(L.lib, name)(None)
    assert L.lib.emt_hinv_tree(None) is None


def test_binding_rejects_host_short_or_wrong_type_buffers(L):
    # a host tensor, a float32 tensor, a strided view or a short buffer never reaches the library
    # as a device address (checked without a GPU: the host-tensor check comes first)
    import torch

    class FakeHInv:
        h, n = None, 8

    with pytest.raises(ValueError, match="CUDA tensor"):
        L.emt_apply(FakeHInv(), torch.zeros(8, dtype=torch.float64), torch.zeros(8, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA tensor"):
        L.emt_apply_noalloc(FakeHInv(), torch.zeros(8, dtype=torch.float64), None)

    class FakeSim:
        h, n, nrhs, n_mon = None, 8, 2, 3

    with pytest.raises(ValueError, match="CUDA tensor"):
        L.emt_step(FakeSim(), 10, torch.zeros(10, 2, 3, dtype=torch.float64))
    assert L._ptr(None) is None and L._ptr(1234) == 1234

    class FakeCuda:   # stands in for a CUDA tensor's attributes
        is_cuda = True

        def __init__(self, dtype, n, contiguous=True):
            self.dtype, self.n, self.c = dtype, n, contiguous

        def numel(self):
            return self.n

        def is_contiguous(self):
            return self.c

        def data_ptr(self):
            return 4096

    assert L._ptr(FakeCuda(torch.float64, 10), 10) == 4096
    with pytest.raises(ValueError, match="float64"):
        L._ptr(FakeCuda(torch.float32, 10), 10)
    with pytest.raises(ValueError, match="contiguous"):
        L._ptr(FakeCuda(torch.float64, 10, contiguous=False), 10)
    with pytest.raises(ValueError, match="elements"):
        L._ptr(FakeCuda(torch.float64, 9), 10, "record_dev")
