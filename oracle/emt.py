"""EMT time stepping (oracle; test infrastructure).

Each step solves Eq. 1 as Eq. 2, v(t) = G^{-1} (i_in(t) + i_his(t - dt)),
then updates every element's history source from v(t) (companion.py).
Readings where the paper is silent: all voltages, currents and history
sources start at zero and the sources are first evaluated at t = dt; a line
trip at step k opens the branch instantaneously before step k is solved (its
conductance leaves G, its current and history are zeroed); a bus fault is a
resistor R_f to ground switched in at step k_on and out at step k_off. Each
switching is its own change of G (Sec. IV): switching in adds 1/R_f e_a e_a^T,
switching out subtracts it again (delta = -1/R_f), so changes made while the
fault is on (a trip, a fault at another bus, a second fault at the same bus)
stay in G after it clears. Several faults on at one bus clear in the order
they were switched in.

The solver is one of: "dense" (Cholesky, refactored on every change),
"exact" (the exact hierarchical store, rebuilt on every change), "paper"
(the approximate store of Algorithm 1, modified by Algorithm 2).
"""
from __future__ import annotations

import numpy as np

from . import companion as cm
from . import dense as _dense
from . import hinv as _hinv
from . import modify as _modify
from . import partition as _part

TRIP = 0
FAULT_ON = 1
FAULT_OFF = 2


class Network:
    """Element data, conductance graph (Eq. 1's G, Sec. II) and partition tree (Sec. III-B) of
    one network at a given dt."""

    def __init__(self, net: dict, dt: float, levels: int = 0, d_th: int = 0, want_tree: bool = True):
        self.net = net
        self.dt = dt
        self.el = cm.elements(net, dt)
        self.gr = cm.graph(net, dt)
        self.G = cm.assemble_dense(self.gr)
        nb = self.el["n_series"]
        self.series_frm = np.asarray(net["br_a"], np.int64)
        self.series_to = np.asarray(net["br_b"], np.int64)
        self.g_series = self.el["g"][:nb].copy()
        self.tree = None
        if want_tree:
            self.tree = _part.build_tree(net["n_bus"], self.series_frm, self.series_to, levels, d_th)


class _Solver:
    """Eq. 2's v = G^{-1} i with one of the three solvers of the module header, and the change
    of G at an event: refactor, rebuild, or Algorithm 2 (Sec. IV)."""

    def __init__(self, nw: Network, kind: str):
        self.nw = nw
        self.kind = kind
        self.G = nw.G.copy()
        if kind == "dense":
            self.s = _dense.DenseSolver(self.G)
        else:
            mode = _hinv.EXACT if kind == "exact" else _hinv.PAPER
            self.s = _hinv.HInv(self.G, nw.tree, nw.g_series, mode)

    def solve(self, rhs):
        """v = G^{-1} rhs (Eq. 2)."""
        return self.s.solve(rhs) if self.kind == "dense" else self.s.apply(rhs)

    def change(self, a, b, delta):
        """G' = G + delta u u^T (Sec. IV) and the matching change of the solver."""
        self.G = _modify.modified_G(self.G, a, b, delta)
        if self.kind == "dense":
            self.s = _dense.DenseSolver(self.G)
        elif self.kind == "exact":
            self.s = _modify.rebuild(self.s, self.nw.series_frm, self.nw.series_to, a, b, delta)
        else:
            self.s = _modify.algorithm2(self.s, self.nw.series_frm, self.nw.series_to, a, b, delta)


def simulate(nw: Network, nsteps: int, events=(), solver: str = "dense", monitor=None,
             src_scale=None, load_scale=None, first_step: int = 1, init=None):
    """Run nsteps steps of Eq. 1 solved as Eq. 2 (Sec. II), with the events and readings of the
    module header; return v at the monitored buses per step [nsteps, n_mon] (all buses when
    monitor is None) and the final state dict."""
    net, el = nw.net, nw.el
    n = net["n_bus"]
    ne = len(el["g"])
    Ih = np.zeros(ne) if init is None else np.array(init["Ih"], float)
    active = np.ones(ne, bool) if init is None else np.array(init["active"], bool)
    sol = _Solver(nw, solver)
    if init is not None:
        for e in np.flatnonzero(~active):
            sol.change(int(el["a"][e]), int(el["b"][e]), -float(el["g"][e]))
    mon = np.arange(n) if monitor is None else np.asarray(monitor, np.int64)
    out = np.zeros((nsteps, len(mon)))
    ev = sorted(events, key=lambda x: x[0])
    faults = {}          # bus -> R_f of the faults on there, in the order they were switched in
    ei = 0
    v = np.zeros(n)
    cur = np.zeros(ne)
    for s in range(nsteps):
        step = first_step + s
        while ei < len(ev) and ev[ei][0] == step:
            _, kind, target, value = ev[ei]
            if kind == TRIP:
                e = int(target)
                a, b = int(el["a"][e]), int(el["b"][e])
                if active[e]:
                    sol.change(a, b, -float(el["g"][e]))
                    active[e] = False
                    Ih[e] = 0.0
            elif kind == FAULT_ON:
                faults.setdefault(int(target), []).append(float(value))
                sol.change(int(target), -1, 1.0 / float(value))
            elif kind == FAULT_OFF:
                on = faults.get(int(target), [])
                if not on:
                    raise ValueError(f"fault switched out at bus {int(target)} where none is on")
                sol.change(int(target), -1, -1.0 / on.pop(0))
            ei += 1
        t = step * nw.dt
        rhs = cm.source_injection(net, t, src_scale, load_scale) + cm.history_injection(el, Ih, n)
        v = sol.solve(rhs)
        cur, Ih = cm.update_history(el, v, Ih, active)
        out[s] = v[mon]
    return out, dict(v=v, Ih=Ih, cur=cur, active=active)
