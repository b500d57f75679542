"""Trapezoidal companion models and nodal assembly (oracle; test infrastructure).

The paper states the EMT network equation G v(t) = i_in(t) + i_his(t - dt)
(Sec. II, Eq. 1) and says it comes from the nodal formulation discretised by
numerical integration (it cites the EMTP book). The trapezoidal companion
model of each element is written here from that rule:

  series RL  v = R i + L di/dt     ->  i(t) = g v_e(t) + I_h,   g = 1/(R + 2L/dt),
                                       I_h <- g [v_e + (2L/dt - R) i]
  series RC  v = R i + v_C, C dv_C/dt = i
                                   ->  i(t) = g v_e(t) + I_h,   g = 1/(R + dt/(2C)),
                                       I_h <- -g [v_e + (dt/(2C) - R) i]
  shunt C    i = C dv/dt           ->  i(t) = g v(t) + I_h,     g = 2C/dt,
                                       I_h <- -(g v + i)
  source     Thevenin e(t), R_s    ->  conductance 1/R_s to ground, injection e(t)/R_s
  load       current sink A sin(w t + phi) leaving the bus

Every history-carrying element is kept in one uniform form: endpoints (a, b)
with b = -1 for ground, conductance g, and the update I_h <- alpha v_e + beta i.
Current i_e flows from a to b, so its history term enters the right-hand side
as -I_h at a and +I_h at b (the sign convention of Eq. 1's i_his).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

KIND_RL = 0
KIND_RC = 1


def elements(net: dict, dt: float) -> dict:
    """History elements of Eq. 1's i_his (Sec. II), with the trapezoidal companion models of the
    module header: series branches first (ids 0..nb-1), then one shunt capacitor per bus.
    Returns endpoints, g, alpha, beta."""
    nb = len(net["br_a"])
    n = net["n_bus"]
    a = np.concatenate([net["br_a"], np.arange(n)]).astype(np.int64)
    b = np.concatenate([net["br_b"], -np.ones(n, np.int64)]).astype(np.int64)
    g = np.zeros(nb + n)
    alpha = np.zeros(nb + n)
    beta = np.zeros(nb + n)
    for e in range(nb):
        R = float(net["R"][e])
        if net["kind"][e] == KIND_RL:
            x = 2.0 * float(net["L"][e]) / dt
            g[e] = 1.0 / (R + x)
            alpha[e] = g[e]
            beta[e] = g[e] * (x - R)
        else:
            x = dt / (2.0 * float(net["C"][e]))
            g[e] = 1.0 / (R + x)
            alpha[e] = -g[e]
            beta[e] = -g[e] * (x - R)
    for n_ in range(n):
        gc = 2.0 * float(net["shunt_C"][n_]) / dt
        g[nb + n_] = gc
        alpha[nb + n_] = -gc
        beta[nb + n_] = -1.0
    return dict(a=a, b=b, g=g, alpha=alpha, beta=beta, n_series=nb)


def graph(net: dict, dt: float) -> dict:
    """The conductance graph of Eq. 1's G (Sec. II): every element and every source conductance
    as a branch (to = -1 for ground). This is the list G is assembled from."""
    el = elements(net, dt)
    src_g = 1.0 / np.asarray(net["src_Rs"], float)
    return dict(n_bus=net["n_bus"],
                frm=np.concatenate([el["a"], np.asarray(net["src_bus"], np.int64)]),
                to=np.concatenate([el["b"], -np.ones(len(src_g), np.int64)]),
                g=np.concatenate([el["g"], src_g]),
                n_series=el["n_series"])


def coupled_rl_admittance(R: float, L: float, L_mut: float, dt: float) -> np.ndarray:
    """Trapezoidal companion admittance of a three-phase RL branch with self inductance L and
    mutual inductance L_mut between any two phases: i = Y v_e + I_h with
    Y = (R I + (2/dt) L3)^-1, L3 = L I + L_mut (J - I) (the single-phase rule of Sec. II applied
    to the coupled inductance matrix)."""
    L3 = L * np.eye(3) + L_mut * (np.ones((3, 3)) - np.eye(3))
    return np.linalg.inv(R * np.eye(3) + (2.0 / dt) * L3)


def three_phase_graph(net: dict, dt: float) -> dict:
    """Conductance graph of a three-phase network (three nodes per bus, Sec. III-A after Eq. 3),
    node = 3 bus + phase. An RL branch's term
    Y (x) (e_a - e_b)(e_a - e_b)^T is split into node branches: a_p-b_p with Y_pp, a_p-b_q
    (p != q) with Y_pq, a_p-a_q and b_p-b_q (p < q) with -Y_pq (zero terms dropped). RC
    branches, shunt capacitors and sources act on each phase alone."""
    frm, to, g = [], [], []
    n = net["n_bus"]
    for e in range(len(net["br_a"])):
        a, b = int(net["br_a"][e]), int(net["br_b"][e])
        if net["kind"][e] == KIND_RL:
            Y = coupled_rl_admittance(float(net["R"][e]), float(net["L"][e]), float(net["L_mut"][e]), dt)
            for p in range(3):
                frm.append(3 * a + p); to.append(3 * b + p); g.append(Y[p, p])
            for p in range(3):
                for q in range(3):
                    if p != q and Y[p, q] != 0.0:
                        frm.append(3 * a + p); to.append(3 * b + q); g.append(Y[p, q])
            for p in range(3):
                for q in range(p + 1, 3):
                    if Y[p, q] != 0.0:
                        frm.append(3 * a + p); to.append(3 * a + q); g.append(-Y[p, q])
                        frm.append(3 * b + p); to.append(3 * b + q); g.append(-Y[p, q])
        else:
            gc = 1.0 / (float(net["R"][e]) + dt / (2.0 * float(net["C"][e])))
            for p in range(3):
                frm.append(3 * a + p); to.append(3 * b + p); g.append(gc)
    for i in range(n):
        for p in range(3):
            frm.append(3 * i + p); to.append(-1); g.append(2.0 * float(net["shunt_C"][i]) / dt)
    for k in range(len(net["src_bus"])):
        for p in range(3):
            frm.append(3 * int(net["src_bus"][k]) + p); to.append(-1); g.append(1.0 / float(net["src_Rs"][k]))
    return dict(n_bus=3 * n, frm=np.asarray(frm, np.int64), to=np.asarray(to, np.int64), g=np.asarray(g, float))


def assemble_dense(gr: dict) -> np.ndarray:
    """G of Eq. 1 (Sec. II) as a dense matrix: the sum over branches of g u u^T, u = e_a - e_b
    (or e_a to ground)."""
    n = gr["n_bus"]
    G = np.zeros((n, n))
    for a, b, g in zip(gr["frm"], gr["to"], gr["g"]):
        G[a, a] += g
        if b >= 0:
            G[b, b] += g
            G[a, b] -= g
            G[b, a] -= g
    return G


def assemble_sparse(gr: dict) -> sp.csc_matrix:
    """G of Eq. 1 (Sec. II) in CSC form, the same sum as assemble_dense."""
    n = gr["n_bus"]
    rows, cols, vals = [], [], []
    for a, b, g in zip(gr["frm"], gr["to"], gr["g"]):
        rows.append(a); cols.append(a); vals.append(g)
        if b >= 0:
            rows += [b, a, b]; cols += [b, b, a]; vals += [g, -g, -g]
    return sp.csc_matrix((vals, (rows, cols)), shape=(n, n))


def source_injection(net: dict, t: float, src_scale=None, load_scale=None) -> np.ndarray:
    """i_in(t) of Eq. 1 (Sec. II): Norton currents e(t)/R_s of the sources minus the load sinks."""
    n = net["n_bus"]
    w = 2.0 * np.pi * net["freq"]
    i = np.zeros(n)
    vm = np.asarray(net["src_Vm"], float) * (1.0 if src_scale is None else np.asarray(src_scale, float))
    np.add.at(i, np.asarray(net["src_bus"]), vm * np.sin(w * t + np.asarray(net["src_phi"])) / np.asarray(net["src_Rs"]))
    if len(net["load_bus"]):
        am = np.asarray(net["load_amp"], float) * (1.0 if load_scale is None else np.asarray(load_scale, float))
        np.add.at(i, np.asarray(net["load_bus"]), -am * np.sin(w * t + np.asarray(net["load_phi"])))
    return i


def history_injection(el: dict, Ih: np.ndarray, n_bus: int) -> np.ndarray:
    """i_his of Eq. 1 (Sec. II): -I_h at the from-bus and +I_h at the to-bus of every element."""
    i = np.zeros(n_bus)
    np.add.at(i, el["a"], -Ih)
    m = el["b"] >= 0
    np.add.at(i, el["b"][m], Ih[m])
    return i


def branch_voltage(el: dict, v: np.ndarray) -> np.ndarray:
    """v_e = v_a - v_b of every element (v_b = 0 for ground), the companion models' input."""
    vb = np.where(el["b"] >= 0, v[np.maximum(el["b"], 0)], 0.0)
    return v[el["a"]] - vb


def update_history(el: dict, v: np.ndarray, Ih: np.ndarray, active: np.ndarray):
    """Element currents at t and the history sources for t + dt: the trapezoidal update
    I_h <- alpha v_e + beta i of the module header (Sec. II, Eq. 1's i_his)."""
    ve = branch_voltage(el, v)
    cur = np.where(active, el["g"] * ve + Ih, 0.0)
    Ih_new = np.where(active, el["alpha"] * ve + el["beta"] * cur, 0.0)
    return cur, Ih_new
