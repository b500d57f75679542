"""Seeded synthetic EMT networks shaped like the paper's workloads.

The paper measures on the 179-bus WECC system and on arrays of copies of it
(Section V, "Case Study"); that data set is not available here, so these
generators stand in for it. They produce raw element data only -- bus
coordinates, branch endpoints, R/L/C values, source and load parameters,
event choices. They hold none of the method's arithmetic: no companion
conductances, no matrix assembly, no partitioning. Both the CPU oracle and the
GPU library consume these arrays and each does its own arithmetic.

Recipe (one 179-bus tile, seed s):
  * 179 points uniform on [0,1]^2.
  * Branches: the Euclidean minimum spanning tree of the Delaunay graph, then
    the shortest remaining Delaunay edges until there are 260 branches
    (planar, mean degree ~2.9).
  * Each branch is series RL with probability 0.9, else series RC;
    R ~ U[0.5, 5] ohm, L ~ U[1, 50] mH, series C ~ U[0.1, 2] uF.
  * Every bus carries a shunt capacitor C ~ U[0.1, 2] uF.
  * 29 distinct buses are Thevenin sine sources e(t) = Vm sin(2 pi 60 t + phi),
    Vm ~ U[0.95, 1.05], phi ~ U[-pi/6, pi/6], Rs ~ U[0.5, 2] ohm.
Tiled arrays place tiles on a rows x cols grid (tile t has seed
1_000_000 + t) and join each grid-adjacent pair with U{3..5} RL tie lines
between buses drawn from the 10 buses nearest the shared border on each side.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import Delaunay
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import minimum_spanning_tree

KIND_RL = 0
KIND_RC = 1

TILE_BUS = 179
TILE_BRANCH = 260
TILE_SRC = 29
FREQ_HZ = 60.0


def _delaunay_edges(pts):
    tri = Delaunay(pts)
    e = set()
    for s in tri.simplices:
        s = sorted(int(v) for v in s)
        e.add((s[0], s[1]))
        e.add((s[0], s[2]))
        e.add((s[1], s[2]))
    e = np.array(sorted(e), dtype=np.int64)
    d = np.hypot(*(pts[e[:, 0]] - pts[e[:, 1]]).T)
    return e, d


def tile(seed: int, n_bus: int = TILE_BUS, n_branch: int = TILE_BRANCH, n_src: int = TILE_SRC) -> dict:
    """One seeded planar tile (raw element data, bus ids 0..n_bus-1)."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n_bus, 2))
    e, d = _delaunay_edges(pts)
    w = coo_matrix((d, (e[:, 0], e[:, 1])), shape=(n_bus, n_bus))
    mst = minimum_spanning_tree(w).tocoo()
    in_mst = set()
    for a, b in zip(mst.row, mst.col):
        in_mst.add((min(int(a), int(b)), max(int(a), int(b))))
    chosen = [(a, b) for a, b in map(tuple, e.tolist()) if (a, b) in in_mst]
    rest = [(float(dd), int(a), int(b)) for (a, b), dd in zip(e.tolist(), d.tolist()) if (a, b) not in in_mst]
    rest.sort()
    need = n_branch - len(chosen)
    chosen += [(a, b) for _, a, b in rest[:max(need, 0)]]
    chosen.sort()
    br = np.array(chosen, dtype=np.int64)
    nb = len(br)
    kind = np.where(rng.random(nb) < 0.9, KIND_RL, KIND_RC).astype(np.int32)
    R = rng.uniform(0.5, 5.0, nb)
    L = rng.uniform(1e-3, 50e-3, nb)
    C = rng.uniform(0.1e-6, 2e-6, nb)
    L[kind == KIND_RC] = 0.0
    C[kind == KIND_RL] = 0.0
    shunt_C = rng.uniform(0.1e-6, 2e-6, n_bus)
    src_bus = np.sort(rng.choice(n_bus, size=n_src, replace=False)).astype(np.int32)
    src_Vm = rng.uniform(0.95, 1.05, n_src)
    src_phi = rng.uniform(-np.pi / 6, np.pi / 6, n_src)
    src_Rs = rng.uniform(0.5, 2.0, n_src)
    return dict(
        n_bus=n_bus, xy=pts,
        br_a=br[:, 0].astype(np.int32), br_b=br[:, 1].astype(np.int32), kind=kind, R=R, L=L, C=C,
        shunt_C=shunt_C,
        src_bus=src_bus, src_Vm=src_Vm, src_phi=src_phi, src_Rs=src_Rs,
        load_bus=np.zeros(0, np.int32), load_amp=np.zeros(0), load_phi=np.zeros(0),
        freq=FREQ_HZ,
    )


def tiled(rows: int, cols: int, seed0: int = 1_000_000, tie_seed: int = 2_000_000) -> dict:
    """rows x cols array of distinct seeded tiles joined by RL tie lines."""
    tiles = [tile(seed0 + t) for t in range(rows * cols)]
    nb = TILE_BUS
    out = {k: [] for k in ("xy", "br_a", "br_b", "kind", "R", "L", "C", "shunt_C",
                           "src_bus", "src_Vm", "src_phi", "src_Rs")}
    for t, tl in enumerate(tiles):
        r, c = divmod(t, cols)
        off = t * nb
        out["xy"].append(tl["xy"] + np.array([c, r], dtype=float))
        out["br_a"].append(tl["br_a"] + off)
        out["br_b"].append(tl["br_b"] + off)
        for k in ("kind", "R", "L", "C", "src_Vm", "src_phi", "src_Rs"):
            out[k].append(tl[k])
        out["shunt_C"].append(tl["shunt_C"])
        out["src_bus"].append(tl["src_bus"] + off)
    rng = np.random.default_rng(tie_seed)
    xy = np.concatenate(out["xy"])
    ties_a, ties_b = [], []
    for t in range(rows * cols):
        r, c = divmod(t, cols)
        for dr, dc in ((0, 1), (1, 0)):
            r2, c2 = r + dr, c + dc
            if r2 >= rows or c2 >= cols:
                continue
            u = r2 * cols + c2
            pa = xy[t * nb:(t + 1) * nb]
            pb = xy[u * nb:(u + 1) * nb]
            if dc == 1:   # shared vertical border at x = c + 1
                da = np.abs(pa[:, 0] - (c + 1)); db = np.abs(pb[:, 0] - (c + 1))
            else:         # shared horizontal border at y = r + 1
                da = np.abs(pa[:, 1] - (r + 1)); db = np.abs(pb[:, 1] - (r + 1))
            ca = np.argsort(da, kind="stable")[:10]
            cb = np.argsort(db, kind="stable")[:10]
            nt = int(rng.integers(3, 6))
            pick_a = rng.choice(ca, size=nt, replace=False)
            pick_b = rng.choice(cb, size=nt, replace=False)
            for x, y in zip(pick_a, pick_b):
                ties_a.append(t * nb + int(x))
                ties_b.append(u * nb + int(y))
    nt = len(ties_a)
    net = dict(
        n_bus=rows * cols * nb, xy=xy,
        br_a=np.concatenate(out["br_a"] + [np.array(ties_a, np.int64)]).astype(np.int32),
        br_b=np.concatenate(out["br_b"] + [np.array(ties_b, np.int64)]).astype(np.int32),
        kind=np.concatenate(out["kind"] + [np.full(nt, KIND_RL, np.int32)]).astype(np.int32),
        R=np.concatenate(out["R"] + [rng.uniform(0.5, 5.0, nt)]),
        L=np.concatenate(out["L"] + [rng.uniform(1e-3, 50e-3, nt)]),
        C=np.concatenate(out["C"] + [np.zeros(nt)]),
        shunt_C=np.concatenate(out["shunt_C"]),
        src_bus=np.concatenate(out["src_bus"]).astype(np.int32),
        src_Vm=np.concatenate(out["src_Vm"]),
        src_phi=np.concatenate(out["src_phi"]),
        src_Rs=np.concatenate(out["src_Rs"]),
        load_bus=np.zeros(0, np.int32), load_amp=np.zeros(0), load_phi=np.zeros(0),
        freq=FREQ_HZ, n_tie=nt,
    )
    return net


def add_loads(net: dict, frac: float = 0.3, seed: int = 13) -> dict:
    """Sine current-sink loads on a fraction of buses (amplitude U[0.05, 0.2])."""
    rng = np.random.default_rng(seed)
    n = net["n_bus"]
    m = int(round(frac * n))
    bus = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int32)
    out = dict(net)
    out["load_bus"] = bus
    out["load_amp"] = rng.uniform(0.05, 0.2, m)
    out["load_phi"] = rng.uniform(-np.pi, np.pi, m)
    return out


def three_phase(net: dict, frac_lo: float = 0.2, frac_hi: float = 0.4, seed: int = 23) -> dict:
    """The same network with three phases per bus: every RL series branch gets a mutual
    inductance between its phases of U[frac_lo, frac_hi] times its self inductance (RC branches:
    none). Element data only; the store works on 3 nodes per bus."""
    rng = np.random.default_rng(seed)
    out = dict(net)
    frac = rng.uniform(frac_lo, frac_hi, len(net["br_a"]))
    out["L_mut"] = np.where(np.asarray(net["kind"]) == 0, frac * np.asarray(net["L"], float), 0.0)
    out["phases"] = 3
    return out


def scenario_scales(net: dict, nrhs: int, sigma: float = 0.05, seed: int = 13) -> tuple:
    """Per-column multiplicative perturbations (1 + eps), eps ~ N(0, sigma),
    for every source amplitude and every load amplitude."""
    rng = np.random.default_rng(seed + 1)
    src = 1.0 + sigma * rng.standard_normal((nrhs, len(net["src_bus"])))
    load = 1.0 + sigma * rng.standard_normal((nrhs, len(net["load_bus"])))
    return src, load


def pick_branch(net: dict, seed: int = 7) -> int:
    """One branch id chosen by seed (the line-trip event)."""
    return int(np.random.default_rng(seed).integers(len(net["br_a"])))


def pick_branches(net: dict, count: int, seed: int = 11) -> np.ndarray:
    """`count` distinct branch ids chosen by seed (N-1 contingency set)."""
    return np.sort(np.random.default_rng(seed).choice(len(net["br_a"]), size=count, replace=False)).astype(np.int32)


def small_network(n_bus: int, seed: int, extra: int = None, n_src: int = None) -> dict:
    """A tiny seeded network of the same construction (for tests)."""
    if extra is None:
        extra = max(n_bus // 3, 1)
    if n_src is None:
        n_src = max(n_bus // 6, 1)
    if n_bus < 3:
        rng = np.random.default_rng(seed)
        br = np.array([[0, 1]], np.int32) if n_bus == 2 else np.zeros((0, 2), np.int32)
        nb = len(br)
        return dict(n_bus=n_bus, xy=rng.random((n_bus, 2)), br_a=br[:, 0].copy(), br_b=br[:, 1].copy(),
                    kind=np.zeros(nb, np.int32), R=rng.uniform(0.5, 5, nb), L=rng.uniform(1e-3, 50e-3, nb),
                    C=np.zeros(nb), shunt_C=rng.uniform(0.1e-6, 2e-6, n_bus),
                    src_bus=np.array([0], np.int32), src_Vm=np.array([1.0]), src_phi=np.array([0.0]),
                    src_Rs=np.array([1.0]), load_bus=np.zeros(0, np.int32), load_amp=np.zeros(0),
                    load_phi=np.zeros(0), freq=FREQ_HZ)
    max_edges = 3 * n_bus - 6 if n_bus > 3 else 3
    return tile(seed, n_bus=n_bus, n_branch=min(n_bus - 1 + extra, max_edges), n_src=min(n_src, n_bus))


def config_network(cfg: int) -> dict:
    """Networks of the five workloads: 1 -> one tile (179 buses), 2/3 -> 2x4
    tiles (1,432 buses), 4 -> 8x8 tiles with loads (11,456 buses)."""
    if cfg == 1:
        return tile(1_000_000)
    if cfg in (2, 3):
        return tiled(2, 4)
    if cfg == 4:
        return add_loads(tiled(8, 8))
    raise ValueError(cfg)


def random_multigraph(seed: int):
    """Random branch lists (n_bus, from, to) that stress the partition's and the store's
    bookkeeping: parallel branches, a hub joined to a third of the buses (a wide gain range and
    wide cuts), two isolated buses and a second component. Branch endpoints only, no parameters."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(60, 340))
    m = int(n * rng.uniform(1.2, 2.2))
    a = rng.integers(0, n - 5, m)
    b = rng.integers(0, n - 5, m)
    keep = a != b
    a, b = list(a[keep]), list(b[keep])
    for k in range(0, m // 4):          # parallel copies of a quarter of the branches
        a.append(a[k])
        b.append(b[k])
    hub = int(rng.integers(0, n - 5))
    for v in rng.choice(n - 5, n // 3, replace=False):
        if int(v) != hub:
            a.append(hub)
            b.append(int(v))
    a += [n - 4, n - 3]                 # a second component; buses n - 2, n - 1 stay isolated
    b += [n - 3, n - 5]
    return n, np.asarray(a, np.int32), np.asarray(b, np.int32)


def random_network(seed: int, src_frac: float = 0.1, load_frac: float = 0.2) -> dict:
    """A simulation network on random_multigraph(seed): RL (90 %) and RC series branches with
    the tile's parameter ranges, a shunt capacitor on every bus (so every bus, the isolated ones
    included, has a path to ground), Thevenin sources and constant-current loads on random buses."""
    n, a, b = random_multigraph(seed)
    rng = np.random.default_rng(seed + 1000)
    nb = len(a)
    kind = np.where(rng.random(nb) < 0.9, KIND_RL, KIND_RC).astype(np.int32)
    R = rng.uniform(0.5, 5.0, nb)
    L = rng.uniform(1e-3, 50e-3, nb)
    C = rng.uniform(0.1e-6, 2e-6, nb)
    L[kind == KIND_RC] = 0.0
    C[kind == KIND_RL] = 0.0
    n_src = max(1, int(src_frac * n))
    n_load = int(load_frac * n)
    src_bus = np.sort(rng.choice(n, size=n_src, replace=False)).astype(np.int32)
    load_bus = np.sort(rng.choice(n, size=n_load, replace=False)).astype(np.int32)
    return dict(
        n_bus=n, br_a=a, br_b=b, kind=kind, R=R, L=L, C=C,
        shunt_C=rng.uniform(0.1e-6, 2e-6, n),
        src_bus=src_bus, src_Vm=rng.uniform(0.95, 1.05, n_src), src_phi=rng.uniform(-np.pi / 6, np.pi / 6, n_src),
        src_Rs=rng.uniform(0.5, 2.0, n_src),
        load_bus=load_bus, load_amp=rng.uniform(0.01, 0.1, n_load), load_phi=rng.uniform(-np.pi / 3, 0.0, n_load),
        freq=FREQ_HZ,
    )
