"""ctypes binding of libemt_hinv.so (argument marshalling only).

Every function mirrors one entry point of include/emt.h under the same name.
Host arrays are NumPy; device buffers are passed as raw pointers (ints) or as
objects with a ``data_ptr()`` method (torch tensors). Nothing here computes any
part of the method: if the shared library is missing, importing this module
raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libemt_hinv.so")

EMT_OK = 0
EMT_ERR_INVALID = 1
EMT_ERR_NOMEM = 2
EMT_ERR_SINGULAR = 3
EMT_ERR_CUDA = 4
EMT_ERR_TIMEOUT = 5
EMT_ERR_STATE = 6
EMT_ERR_UNSUPPORTED = 7
STATUS_NAMES = {0: "EMT_OK", 1: "EMT_ERR_INVALID", 2: "EMT_ERR_NOMEM", 3: "EMT_ERR_SINGULAR", 4: "EMT_ERR_CUDA",
                5: "EMT_ERR_TIMEOUT", 6: "EMT_ERR_STATE", 7: "EMT_ERR_UNSUPPORTED"}

EMT_MODE_EXACT = 0
EMT_MODE_PAPER = 1
EMT_PREC_FP64 = 0
EMT_PREC_FF64 = 1
EMT_PREC_FP32 = 2
EMT_KIND_RL = 0
EMT_KIND_RC = 1
EMT_EVENT_TRIP = 0
EMT_EVENT_FAULT_ON = 1
EMT_EVENT_FAULT_OFF = 2

_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)


class EmtGraph(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_branch", C.c_int32), ("from_", _i32p), ("to", _i32p), ("g", _f64p)]


class EmtHinvOpts(C.Structure):
    _fields_ = [("levels", C.c_int32), ("d_th", C.c_int32), ("mode", C.c_int32), ("precision", C.c_int32),
                ("nodes_per_bus", C.c_int32)]


class EmtNetwork(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_branch", C.c_int32), ("from_", _i32p), ("to", _i32p), ("kind", _i32p),
                ("R", _f64p), ("L", _f64p), ("C", _f64p), ("shunt_C", _f64p),
                ("n_src", C.c_int32), ("src_bus", _i32p), ("src_Vm", _f64p), ("src_phi", _f64p), ("src_Rs", _f64p),
                ("n_load", C.c_int32), ("load_bus", _i32p), ("load_amp", _f64p), ("load_phi", _f64p),
                ("freq", C.c_double)]


class EmtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"native library not built: {LIB_PATH} (run __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    sigs = {
        "emt_last_error": (C.c_char_p, []),
        "emt_version": (C.c_char_p, []),
        "emt_tree_build": (C.c_int, [C.POINTER(EmtGraph), C.POINTER(EmtHinvOpts), C.POINTER(vp)]),
        "emt_tree_sizes": (C.c_int, [vp, _i32p, _i32p, _i32p]),
        "emt_tree_arrays": (C.c_int, [vp] + [_i32p] * 11),
        "emt_tree_destroy": (None, [vp]),
        "emt_build_hinv": (C.c_int, [C.POINTER(EmtGraph), C.POINTER(EmtHinvOpts), vp, C.POINTER(vp)]),
        "emt_hinv_tree": (vp, [vp]),
        "emt_hinv_get_partition": (C.c_int, [vp, _i32p, _i32p, _i32p, _i32p]),
        "emt_apply": (C.c_int, [vp, vp, vp, C.c_int32, C.c_int64, C.c_int32, C.c_double, vp]),
        "emt_modify_branch": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_double, vp]),
        "emt_hinv_sync": (C.c_int, [vp, vp]),
        "emt_apply_tune": (C.c_int, [vp, C.c_int32, C.c_int32, _i32p]),
        "emt_hinv_destroy": (None, [vp]),
        "emt_sim_create": (C.c_int, [C.POINTER(EmtNetwork), C.POINTER(EmtHinvOpts), C.c_double, C.c_int32, _f64p,
                                     _f64p, vp, C.POINTER(vp)]),
        "emt_sim_schedule": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_int32]),
        "emt_sim_monitor": (C.c_int, [vp, C.c_int32, _i32p]),
        "emt_step": (C.c_int, [vp, C.c_int32, vp, vp]),
        "emt_sim_read": (C.c_int, [vp, C.c_int32, _f64p]),
        "emt_sim_set_rows_per_cta": (C.c_int, [vp, C.c_int32]),
        "emt_sim_destroy": (None, [vp]),
        "emt_sim_reset": (C.c_int, [vp, vp]),
        "emt_sim_stats": (C.c_int, [vp, C.POINTER(C.c_int64), C.c_int32]),
        "emt_sim_bench_kernel": (C.c_int, [vp, C.c_int32, C.c_int32, vp]),
        "emt_apply_noalloc": (C.c_int, [vp, vp, vp, vp]),
        "emt_sim_tune": (C.c_int, [vp, C.c_int32, C.c_int32]),
        "emt_sim_set_inject": (C.c_int, [vp, C.c_int32, C.c_int32]),
        "emt_sim_autotune": (C.c_int, [vp, C.c_int32, _i32p, _i32p, vp]),
        "emt_server_create": (C.c_int, [C.c_int32, C.c_uint64, C.POINTER(vp)]),
        "emt_server_add_network": (C.c_int, [vp, C.POINTER(EmtNetwork), C.POINTER(EmtHinvOpts), C.c_double, C.c_int32,
                                             C.c_int32, _i32p, _i32p]),
        "emt_server_submit": (C.c_int, [vp, C.c_int32, C.c_double, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                        C.c_int32, C.c_int32, _i32p]),
        "emt_server_submit_network": (C.c_int, [vp, C.POINTER(EmtNetwork), C.POINTER(EmtHinvOpts), C.c_double,
                                                C.c_int32, _i32p, C.c_double, C.c_int32, C.c_int32, C.c_int32,
                                                C.c_double, C.c_int32, C.c_int32, _i32p]),
        "emt_server_run": (C.c_int, [vp]),
        "emt_server_result": (C.c_int, [vp, C.c_int32, _f64p, _f64p]),
        "emt_server_stats": (C.c_int, [vp, _f64p, C.c_int32]),
        "emt_server_destroy": (None, [vp]),
        "emt_selftest_bounded_wait": (C.c_int, [C.c_int32, vp]),
        "emt_build_hinv_from_network": (C.c_int, [C.POINTER(EmtNetwork), C.c_double, C.POINTER(EmtHinvOpts), vp,
                                                  C.POINTER(vp)]),
        "emt_build_hinv_from_network3": (C.c_int, [C.POINTER(EmtNetwork), _f64p, C.c_double, C.POINTER(EmtHinvOpts),
                                                   vp, C.POINTER(vp)]),
        "emt_sim3_create": (C.c_int, [C.POINTER(EmtNetwork), _f64p, C.POINTER(EmtHinvOpts), C.c_double, vp,
                                      C.POINTER(vp)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()
EXPORTED = ("emt_last_error", "emt_version", "emt_tree_build", "emt_tree_sizes", "emt_tree_arrays", "emt_tree_destroy",
            "emt_build_hinv", "emt_hinv_tree", "emt_hinv_get_partition", "emt_apply", "emt_modify_branch",
            "emt_hinv_sync", "emt_apply_tune", "emt_hinv_destroy",
            "emt_sim_create", "emt_sim_schedule", "emt_sim_monitor", "emt_step", "emt_sim_read",
            "emt_sim_set_rows_per_cta", "emt_sim_destroy", "emt_sim_reset", "emt_sim_stats",
            "emt_sim_bench_kernel", "emt_apply_noalloc", "emt_sim_tune", "emt_sim_set_inject", "emt_sim_autotune", "emt_server_create",
            "emt_server_add_network", "emt_server_submit", "emt_server_submit_network", "emt_server_run",
            "emt_server_result", "emt_server_stats",
            "emt_server_destroy", "emt_selftest_bounded_wait", "emt_build_hinv_from_network",
            "emt_build_hinv_from_network3", "emt_sim3_create")


def _check(code):
    if code != EMT_OK:
        raise EmtError(code, lib.emt_last_error().decode())


def _ptr(x, n_min=0, what="buffer"):
    """Device address of a CUDA float64 tensor (contiguous, at least n_min elements), checked here so
    that a host tensor or a short buffer is an error in Python, never an address the GPU reads; a raw
    integer address is passed through as the caller's responsibility."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not getattr(x, "is_cuda", False):
            raise ValueError(f"{what}: expected a CUDA tensor, got one on {getattr(x, 'device', 'the host')}")
        if str(getattr(x, "dtype", "")) != "torch.float64":
            raise ValueError(f"{what}: expected float64, got {getattr(x, 'dtype', None)}")
        if not x.is_contiguous():
            raise ValueError(f"{what}: expected a contiguous tensor")
        if x.numel() < n_min:
            raise ValueError(f"{what}: {x.numel()} elements, the call writes or reads {n_min}")
        return x.data_ptr()
    raise TypeError("expected a device pointer or an object with data_ptr()")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream   # torch.cuda.Stream


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None and a.size else None


def make_graph(n_bus, frm, to, g):
    keep = [_i32(frm), _i32(to), _f64(g)]
    gr = EmtGraph(int(n_bus), len(keep[0]), _p(keep[0], _i32p), _p(keep[1], _i32p), _p(keep[2], _f64p))
    return gr, keep


def make_opts(levels=0, d_th=0, mode=EMT_MODE_EXACT, precision=EMT_PREC_FP64, nodes_per_bus=0):
    return EmtHinvOpts(int(levels), int(d_th), int(mode), int(precision), int(nodes_per_bus))


def make_network(net: dict):
    """emt_network from the raw element dict of the synthetic generator."""
    k = dict(frm=_i32(net["br_a"]), to=_i32(net["br_b"]), kind=_i32(net["kind"]), R=_f64(net["R"]),
             L=_f64(net["L"]), C=_f64(net["C"]), shunt=_f64(net["shunt_C"]), sb=_i32(net["src_bus"]),
             sv=_f64(net["src_Vm"]), sp=_f64(net["src_phi"]), sr=_f64(net["src_Rs"]), lb=_i32(net["load_bus"]),
             la=_f64(net["load_amp"]), lp=_f64(net["load_phi"]))
    nw = EmtNetwork(int(net["n_bus"]), len(k["frm"]), _p(k["frm"], _i32p), _p(k["to"], _i32p), _p(k["kind"], _i32p),
                    _p(k["R"], _f64p), _p(k["L"], _f64p), _p(k["C"], _f64p), _p(k["shunt"], _f64p),
                    len(k["sb"]), _p(k["sb"], _i32p), _p(k["sv"], _f64p), _p(k["sp"], _f64p), _p(k["sr"], _f64p),
                    len(k["lb"]), _p(k["lb"], _i32p), _p(k["la"], _f64p), _p(k["lp"], _f64p),
                    float(net["freq"]))
    return nw, k


# ------------------------------------------------------------------ entry points (same names)
def emt_version():
    return lib.emt_version().decode()


def emt_tree_build(n_bus, frm, to, g=None, levels=0, d_th=0, nodes_per_bus=0):
    if g is None:
        g = np.ones(len(frm))
    gr, keep = make_graph(n_bus, frm, to, g)
    o = make_opts(levels, d_th, nodes_per_bus=nodes_per_bus)
    h = C.c_void_p()
    _check(lib.emt_tree_build(C.byref(gr), C.byref(o), C.byref(h)))
    try:
        return tree_arrays(h.value, n_bus)
    finally:
        lib.emt_tree_destroy(h)


def tree_arrays(handle, n_bus):
    nn, nl, nc = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib.emt_tree_sizes(handle, C.byref(nn), C.byref(nl), C.byref(nc)))
    nn, nl, nc = nn.value, nl.value, nc.value
    out = {k: np.zeros(s, np.int32) for k, s in
           (("perm", n_bus), ("lo", nn), ("hi", nn), ("parent", nn), ("left", nn), ("right", nn), ("depth", nn),
            ("cut_ptr", nn + 1), ("cut_a", nc), ("cut_b", nc), ("cut_e", nc))}
    _check(lib.emt_tree_arrays(handle, *[_p(out[k], _i32p) if out[k].size else None for k in
                                         ("perm", "lo", "hi", "parent", "left", "right", "depth", "cut_ptr", "cut_a",
                                          "cut_b", "cut_e")]))
    return out


class HInv:
    """Owning wrapper of an emt_hinv handle."""

    def __init__(self, handle, n_bus):
        self.h = handle
        self.n = n_bus

    def __del__(self):
        if getattr(self, "h", None):
            lib.emt_hinv_destroy(self.h)
            self.h = None

    def tree(self):
        return tree_arrays(lib.emt_hinv_tree(self.h), self.n)


def emt_hinv_get_partition(h: HInv):
    """(perm, node_lo, node_hi, parent) of the handle's partition tree."""
    nn = C.c_int32()
    _check(lib.emt_tree_sizes(lib.emt_hinv_tree(h.h), C.byref(nn), None, None))
    perm = np.zeros(h.n, np.int32)
    lo, hi, parent = (np.zeros(nn.value, np.int32) for _ in range(3))
    _check(lib.emt_hinv_get_partition(h.h, *[_p(a, _i32p) for a in (perm, lo, hi, parent)]))
    return perm, lo, hi, parent


def emt_build_hinv(n_bus, frm, to, g, levels=0, d_th=0, mode=EMT_MODE_EXACT, precision=EMT_PREC_FP64, stream=None,
                   nodes_per_bus=0):
    gr, keep = make_graph(n_bus, frm, to, g)
    o = make_opts(levels, d_th, mode, precision, nodes_per_bus)
    h = C.c_void_p()
    _check(lib.emt_build_hinv(C.byref(gr), C.byref(o), _stream(stream), C.byref(h)))
    return HInv(h.value, n_bus)


def emt_apply(h: HInv, i_dev, v_dev, nrhs=1, ld=None, max_refine=0, tol=0.0, stream=None):
    ld = int(ld if ld is not None else h.n)
    need = ld * (int(nrhs) - 1) + h.n if int(nrhs) >= 1 else 0
    _check(lib.emt_apply(h.h, _ptr(i_dev, need, "i_dev"), _ptr(v_dev, need, "v_dev"), int(nrhs), ld,
                         int(max_refine), float(tol), _stream(stream)))


def emt_apply_noalloc(h: HInv, i_dev, v_dev, stream=None):
    """Single-vector apply that allocates nothing (scratch in a fixed device array)."""
    _check(lib.emt_apply_noalloc(h.h, _ptr(i_dev, h.n, "i_dev"), _ptr(v_dev, h.n, "v_dev"), _stream(stream)))


def emt_modify_branch(h: HInv, bus_a, bus_b, delta_g, stream=None):
    _check(lib.emt_modify_branch(h.h, int(bus_a), int(bus_b), float(delta_g), _stream(stream)))


def emt_apply_tune(h: HInv, kernels=0, warps=0):
    """Kernels of the single-vector apply on large stores; returns what the next apply runs
    (2 single launch, 1 three kernels, 0 small-store kernels or no plan yet)."""
    used = C.c_int32(-1)
    _check(lib.emt_apply_tune(h.h, int(kernels), int(warps), C.byref(used)))
    return int(used.value)


def emt_hinv_sync(h: HInv, stream=None):
    _check(lib.emt_hinv_sync(h.h, _stream(stream)))


class Sim:
    """Owning wrapper of an emt_sim handle."""

    def __init__(self, handle, n_bus, nrhs):
        self.h = handle
        self.n = n_bus
        self.nrhs = nrhs
        self.n_mon = 0

    def __del__(self):
        if getattr(self, "h", None):
            lib.emt_sim_destroy(self.h)
            self.h = None


def emt_sim_create(net: dict, dt, levels=0, d_th=0, mode=EMT_MODE_EXACT, precision=EMT_PREC_FF64, nrhs=1,
                   src_scale=None, load_scale=None, stream=None):
    nw, keep = make_network(net)
    o = make_opts(levels, d_th, mode, precision)
    ss = _f64(src_scale) if src_scale is not None else None
    ls = _f64(load_scale) if load_scale is not None else None
    h = C.c_void_p()
    _check(lib.emt_sim_create(C.byref(nw), C.byref(o), float(dt), int(nrhs), _p(ss, _f64p), _p(ls, _f64p),
                              _stream(stream), C.byref(h)))
    return Sim(h.value, int(net["n_bus"]), nrhs)


def emt_sim_schedule(s: Sim, step, kind, target, value=0.0, column=-1):
    _check(lib.emt_sim_schedule(s.h, int(step), int(kind), int(target), float(value), int(column)))


def emt_sim_monitor(s: Sim, buses):
    b = _i32(buses)
    _check(lib.emt_sim_monitor(s.h, len(b), _p(b, _i32p)))
    s.n_mon = len(b)


def emt_step(s: Sim, n_steps, record_dev=None, stream=None):
    need = max(int(n_steps), 0) * s.nrhs * s.n_mon
    _check(lib.emt_step(s.h, int(n_steps), _ptr(record_dev, need, "record_dev"), _stream(stream)))


def emt_sim_read(s: Sim, what=0):
    out = np.zeros(s.n * s.nrhs if what == 0 else 1)
    _check(lib.emt_sim_read(s.h, int(what), _p(out, _f64p)))
    return out


def emt_sim_set_rows_per_cta(s: Sim, rows):
    _check(lib.emt_sim_set_rows_per_cta(s.h, int(rows)))


def emt_sim_reset(s: Sim, stream=None):
    _check(lib.emt_sim_reset(s.h, _stream(stream)))


STAT_KEYS = ("n_bus", "n_leaf", "leaf_elems", "factor_elems", "core_elems", "n_cta", "n_incidence", "n_cut_rows",
             "s_total", "launches", "n_series", "n_elements", "inject_columns_per_thread", "inject_variant",
             "residual_columns_per_thread")


def emt_sim_stats(s: Sim):
    out = (C.c_int64 * len(STAT_KEYS))()
    _check(lib.emt_sim_stats(s.h, out, len(STAT_KEYS)))
    return dict(zip(STAT_KEYS, [int(x) for x in out]))


def emt_sim_bench_kernel(s: Sim, which, reps, stream=None):
    _check(lib.emt_sim_bench_kernel(s.h, int(which), int(reps), _stream(stream)))


def emt_sim_tune(s: Sim, rows_per_cta=0, kernels=2):
    _check(lib.emt_sim_tune(s.h, int(rows_per_cta), int(kernels)))


def emt_sim_set_inject(s: Sim, mode=0, positions_per_cta=0):
    _check(lib.emt_sim_set_inject(s.h, int(mode), int(positions_per_cta)))


def emt_sim_autotune(s: Sim, probe_steps=256, stream=None):
    r, k = C.c_int32(), C.c_int32()
    _check(lib.emt_sim_autotune(s.h, int(probe_steps), C.byref(r), C.byref(k), _stream(stream)))
    return r.value, k.value


class Server:
    """Owning wrapper of an emt_server handle."""

    def __init__(self, handle):
        self.h = handle
        self.n_mon = {}
        self.steps = {}

    def __del__(self):
        if getattr(self, "h", None):
            lib.emt_server_destroy(self.h)
            self.h = None


def emt_server_create(tick_steps=100, hbm_budget_bytes=0):
    h = C.c_void_p()
    _check(lib.emt_server_create(int(tick_steps), int(hbm_budget_bytes), C.byref(h)))
    return Server(h.value)


def emt_server_add_network(srv: Server, net: dict, dt, levels=0, d_th=0, max_slots=64, monitor=None):
    nw, keep = make_network(net)
    o = make_opts(levels, d_th, EMT_MODE_EXACT, EMT_PREC_FP32)
    mon = _i32(monitor if monitor is not None else np.arange(min(16, net["n_bus"])))
    nid = C.c_int32()
    _check(lib.emt_server_add_network(srv.h, C.byref(nw), C.byref(o), float(dt), int(max_slots), len(mon),
                                      _p(mon, _i32p), C.byref(nid)))
    srv.n_mon[nid.value] = len(mon)
    return nid.value


def emt_server_submit(srv: Server, net_id, arrival_s, n_steps, event_kind=-1, target=0, value=0.0, event_step=0,
                      event_len=0):
    rid = C.c_int32()
    _check(lib.emt_server_submit(srv.h, int(net_id), float(arrival_s), int(n_steps), int(event_kind), int(target),
                                 float(value), int(event_step), int(event_len), C.byref(rid)))
    srv.steps[rid.value] = (int(n_steps), int(net_id))
    return rid.value


def emt_server_submit_network(srv: Server, net: dict, dt, arrival_s, n_steps, event_kind=-1, target=0, value=0.0,
                              event_step=0, event_len=0, levels=0, d_th=0, monitor=None):
    nw, keep = make_network(net)
    o = make_opts(levels, d_th, EMT_MODE_EXACT, EMT_PREC_FP32)
    mon = _i32(monitor if monitor is not None else np.arange(min(16, net["n_bus"])))
    rid = C.c_int32()
    _check(lib.emt_server_submit_network(srv.h, C.byref(nw), C.byref(o), float(dt), len(mon), _p(mon, _i32p),
                                         float(arrival_s), int(n_steps), int(event_kind), int(target), float(value),
                                         int(event_step), int(event_len), C.byref(rid)))
    srv.steps[rid.value] = (int(n_steps), ("req", len(mon)))
    return rid.value


def emt_server_run(srv: Server):
    _check(lib.emt_server_run(srv.h))


def emt_server_result(srv: Server, req_id):
    n_steps, nid = srv.steps[req_id]
    n_mon = nid[1] if isinstance(nid, tuple) else srv.n_mon[nid]
    out = np.zeros((n_steps, n_mon))
    times = np.zeros(3)
    _check(lib.emt_server_result(srv.h, int(req_id), _p(out, _f64p), _p(times, _f64p)))
    return out, times


SERVER_STAT_KEYS = ("wall_s", "bus_steps", "bus_steps_per_s", "p50_s", "p99_s", "max_s", "max_queue", "ticks",
                    "finished", "builds", "cache_hits", "build_s", "evictions")


def emt_server_stats(srv: Server):
    out = np.zeros(len(SERVER_STAT_KEYS))
    _check(lib.emt_server_stats(srv.h, _p(out, _f64p), len(out)))
    return dict(zip(SERVER_STAT_KEYS, out.tolist()))


def emt_selftest_bounded_wait(limit_us=1000, stream=None):
    """Returns the status code (EMT_ERR_TIMEOUT expected)."""
    return lib.emt_selftest_bounded_wait(int(limit_us), _stream(stream))


def emt_build_hinv_from_network(net: dict, dt, levels=0, d_th=0, mode=EMT_MODE_EXACT, precision=EMT_PREC_FP64,
                                stream=None):
    nw, keep = make_network(net)
    o = make_opts(levels, d_th, mode, precision)
    h = C.c_void_p()
    _check(lib.emt_build_hinv_from_network(C.byref(nw), float(dt), C.byref(o), _stream(stream), C.byref(h)))
    return HInv(h.value, int(net["n_bus"]))


def emt_build_hinv_from_network3(net: dict, dt, levels=0, d_th=0, mode=EMT_MODE_EXACT, precision=EMT_PREC_FP64,
                                 stream=None, nodes_per_bus=0):
    """Store of a three-phase network (3 nodes per bus; `net["L_mut"]` mutual inductances); block cuts
    unless nodes_per_bus == 1."""
    nw, keep = make_network(net)
    lm = _f64(net["L_mut"])
    o = make_opts(levels, d_th, mode, precision, nodes_per_bus)
    h = C.c_void_p()
    _check(lib.emt_build_hinv_from_network3(C.byref(nw), _p(lm, _f64p), float(dt), C.byref(o), _stream(stream),
                                            C.byref(h)))
    return HInv(h.value, 3 * int(net["n_bus"]))


def emt_sim3_create(net: dict, dt, levels=0, d_th=0, mode=EMT_MODE_EXACT, precision=EMT_PREC_FF64, stream=None,
                    nodes_per_bus=0):
    """Three-phase simulation (3 nodes per bus; `net["L_mut"]` mutual inductances of the RL branches);
    block cuts unless nodes_per_bus == 1."""
    nw, keep = make_network(net)
    lm = _f64(net["L_mut"])
    o = make_opts(levels, d_th, mode, precision, nodes_per_bus)
    h = C.c_void_p()
    _check(lib.emt_sim3_create(C.byref(nw), _p(lm, _f64p), C.byref(o), float(dt), _stream(stream), C.byref(h)))
    return Sim(h.value, 3 * int(net["n_bus"]), 1)
