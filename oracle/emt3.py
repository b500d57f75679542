"""Three-phase EMT time stepping (oracle; test infrastructure).

The paper counts three nodes per bus (Sec. III-A, after Eq. 3) but states no three-phase element
model. The readings here, with node = 3 bus + phase:

  * a series RL branch couples its phases through L3 = L I + L_mut (J - I). The trapezoidal rule
    of Sec. II applied to v_e = R i + L3 di/dt, with 3-vectors v_e, i and I_h, gives
        i(t) = Y v_e(t) + I_h,   Y = (R I + (2/dt) L3)^-1,   I_h <- Y [v_e + ((2/dt) L3 - R I) i]
    (companion.coupled_rl_admittance gives Y);
  * series RC branches, shunt capacitors and source resistances act on each phase alone, with
    the single-phase companion models of companion.py;
  * sources and loads are balanced: phase p lags phase 0 by 2 pi p / 3.

A trip opens all three phases of a branch before the step is solved: its terms leave G, and its
currents and histories are zeroed. A fault connects one node (a phase of a bus) to ground through
R_f: FAULT_ON adds (1/R_f) e_x e_x^T to G before its step is solved, FAULT_OFF takes the oldest
fault still on at that node back out (the single-phase semantics of emt.py, node by node; a
three-phase fault is three node faults). G is the node-branch graph of
companion.three_phase_graph.
"""
from __future__ import annotations

import numpy as np

from . import companion as cm
from . import dense as _dense

TRIP = 0
FAULT_ON = 1
FAULT_OFF = 2


def fault_conductance(r_f: float) -> float:
    """The conductance a fault through R_f adds to its node's diagonal of G (Sec. IV's change)."""
    return 1.0 / r_f


def phase_shift(p: int) -> float:
    """Angle of phase p against phase 0 (balanced sequence a, b, c)."""
    return -2.0 * np.pi * p / 3.0


def source_injection3(net: dict, t: float) -> np.ndarray:
    """i_in(t) of Eq. 1 (Sec. II) on the 3 n nodes: per phase, the Norton current e_p(t)/R_s of every
    source minus the load sinks."""
    n = net["n_bus"]
    w = 2.0 * np.pi * net["freq"]
    i = np.zeros(3 * n)
    sb = np.asarray(net["src_bus"], np.int64)
    lb = np.asarray(net["load_bus"], np.int64)
    for p in range(3):
        e = np.asarray(net["src_Vm"], float) * np.sin(w * t + np.asarray(net["src_phi"], float) + phase_shift(p))
        np.add.at(i, 3 * sb + p, e / np.asarray(net["src_Rs"], float))
        if len(lb):
            a = np.asarray(net["load_amp"], float) * np.sin(w * t + np.asarray(net["load_phi"], float) + phase_shift(p))
            np.add.at(i, 3 * lb + p, -a)
    return i


def _branch_block(net: dict, e: int, dt: float) -> np.ndarray:
    """The 3 x 3 admittance a series branch adds between its end buses (Y, or g I for RC)."""
    R = float(net["R"][e])
    if net["kind"][e] == cm.KIND_RL:
        return cm.coupled_rl_admittance(R, float(net["L"][e]), float(net["L_mut"][e]), dt)
    return np.eye(3) / (R + dt / (2.0 * float(net["C"][e])))


def simulate3(net: dict, dt: float, nsteps: int, events=(), monitor=None, init=None, first_step: int = 1):
    """Run nsteps steps of Eq. 1 solved as Eq. 2 (Sec. II) on the three-phase network, with the
    readings of the module header, from rest or from the state `init` of an earlier call; return the
    node voltages per step [nsteps, n_mon] (all 3 n nodes when monitor is None) and the final state."""
    n = net["n_bus"]
    nb = len(net["br_a"])
    a_bus = np.asarray(net["br_a"], np.int64)
    b_bus = np.asarray(net["br_b"], np.int64)
    G = cm.assemble_dense(cm.three_phase_graph(net, dt))
    sol = _dense.DenseSolver(G)
    Y = [_branch_block(net, e, dt) for e in range(nb)]
    # history matrices: RL  I_h <- Y (v_e + H i),  H = (2/dt) L3 - R I;
    #                   RC  I_h <- -g (v_e + (dt/(2C) - R) i)  (a multiple of I per phase)
    Hm = []
    for e in range(nb):
        R = float(net["R"][e])
        if net["kind"][e] == cm.KIND_RL:
            L, M = float(net["L"][e]), float(net["L_mut"][e])
            L3 = L * np.eye(3) + M * (np.ones((3, 3)) - np.eye(3))
            Hm.append((2.0 / dt) * L3 - R * np.eye(3))
        else:
            Hm.append((dt / (2.0 * float(net["C"][e])) - R) * np.eye(3))
    gsh = np.repeat(2.0 * np.asarray(net["shunt_C"], float) / dt, 3)
    Ih = np.zeros((nb, 3))
    cur = np.zeros((nb, 3))
    Ih_sh = np.zeros(3 * n)
    active = np.ones(nb, bool)

    def open_branch(e):
        A, B = 3 * a_bus[e], 3 * b_bus[e]
        G[A:A + 3, A:A + 3] -= Y[e]
        G[B:B + 3, B:B + 3] -= Y[e]
        G[A:A + 3, B:B + 3] += Y[e]
        G[B:B + 3, A:A + 3] += Y[e]

    if init is not None:
        Ih, cur = np.array(init["Ih"], float), np.array(init["cur"], float)
        Ih_sh, active = np.array(init["Ih_sh"], float), np.array(init["active"], bool)
        for e in np.flatnonzero(~active):
            open_branch(e)
        sol = _dense.DenseSolver(G)
    mon = np.arange(3 * n) if monitor is None else np.asarray(monitor, np.int64)
    out = np.zeros((nsteps, len(mon)))
    ev = sorted(events, key=lambda x: x[0])
    ei = 0
    v = np.zeros(3 * n)
    faults = {} if init is None else {int(k): list(x) for k, x in init.get("faults", {}).items()}
    for x, rs in faults.items():
        for r in rs:
            G[x, x] += fault_conductance(r)
    if faults:
        sol = _dense.DenseSolver(G)
    for s in range(nsteps):
        step = first_step + s
        while ei < len(ev) and ev[ei][0] == step:
            _, kind, target, value = ev[ei]
            if kind == TRIP and active[int(target)]:
                e = int(target)
                open_branch(e)
                sol = _dense.DenseSolver(G)
                active[e] = False
                Ih[e] = 0.0
                cur[e] = 0.0
            elif kind == FAULT_ON:
                x = int(target)
                faults.setdefault(x, []).append(float(value))
                G[x, x] += fault_conductance(float(value))
                sol = _dense.DenseSolver(G)
            elif kind == FAULT_OFF:
                x = int(target)
                if not faults.get(x):
                    raise ValueError(f"FAULT_OFF at node {x} with no fault on")
                G[x, x] -= fault_conductance(faults[x].pop(0))
                sol = _dense.DenseSolver(G)
            ei += 1
        rhs = source_injection3(net, step * dt) - Ih_sh
        for e in np.flatnonzero(active):
            A, B = 3 * a_bus[e], 3 * b_bus[e]
            rhs[A:A + 3] -= Ih[e]
            rhs[B:B + 3] += Ih[e]
        v = sol.solve(rhs)
        for e in np.flatnonzero(active):
            A, B = 3 * a_bus[e], 3 * b_bus[e]
            ve = v[A:A + 3] - v[B:B + 3]
            cur[e] = Y[e] @ ve + Ih[e]
            if net["kind"][e] == cm.KIND_RL:
                Ih[e] = Y[e] @ (ve + Hm[e] @ cur[e])
            else:
                Ih[e] = -(Y[e] @ (ve + Hm[e] @ cur[e]))
        i_sh = gsh * v + Ih_sh
        Ih_sh = -gsh * v - i_sh
        out[s] = v[mon]
    return out, dict(v=v, cur=cur, Ih=Ih, Ih_sh=Ih_sh, active=active, faults=faults)
