"""Inverse modification after a network change (oracle; test infrastructure).

Sec. IV of the paper. A change between buses a and b (a line trip, a fault
branch) or at one bus (a fault to ground) is G' = G + delta u u^T with
u = e_a - e_b, or u = e_a for a bus-to-ground change.

  * explicit recomputation: rebuild the store from G' (the reference every
    local update is compared with);
  * Sherman-Morrison closed form of the exact inverse (dense.sherman_morrison);
  * Algorithm 2 (Modification / UpdateM): find the lowest common ancestor
    (LCA) of the leaves holding a and b, directly re-invert the touched
    leaves, and recompute the factors of Eq. 9 on the two paths up to the
    LCA; everything else is kept. `to_root=True` continues the same
    recomputation up to the root (then it equals a rebuild).

The conductance change is carried by the lowest-id series branch joining a
and b (its g becomes g + delta); a cross-leaf change needs such a branch,
because the tree's cut lists are fixed at build time.
"""
from __future__ import annotations

import copy

import numpy as np

from . import dense as _dense
from .hinv import HInv, EXACT, PAPER
from .partition import leaf_of, lca


def find_branch(frm, to, a: int, b: int) -> int:
    """The lowest-id series branch joining a and b (-1 if none): the branch a change between two
    buses is carried by (module header)."""
    for e, (x, y) in enumerate(zip(frm, to)):
        if (int(x) == a and int(y) == b) or (int(x) == b and int(y) == a):
            return e
    return -1


def modified_G(G: np.ndarray, a: int, b: int, delta: float) -> np.ndarray:
    """G' = G + delta u u^T for a change between a and b, or at a alone when b < 0 (Sec. IV)."""
    G = np.array(G, float)
    G[a, a] += delta
    if b >= 0:
        G[b, b] += delta
        G[a, b] -= delta
        G[b, a] -= delta
    return G


def u_vector(n: int, a: int, b: int) -> np.ndarray:
    """u = e_a - e_b, or e_a for a change to ground (Sec. IV)."""
    u = np.zeros(n)
    u[a] = 1.0
    if b >= 0:
        u[b] = -1.0
    return u


def touched_path(tree: dict, a_pos: int, b_pos: int, to_root: bool):
    """Algorithm 2's touched set (Sec. IV): the leaves holding a and b, re-inverted, and the
    internal nodes on their paths up to the lowest common ancestor (to the root when to_root),
    recomputed children first."""
    la = leaf_of(tree, a_pos)
    lb = leaf_of(tree, b_pos) if b_pos >= 0 else la
    top = lca(tree, la, lb)
    leaves = sorted({la, lb})
    nodes = set()
    for leaf in leaves:
        x = leaf
        while True:
            if tree["left"][x] >= 0:
                nodes.add(x)
            if x == top and not to_root:
                break
            if tree["parent"][x] < 0:
                break
            x = int(tree["parent"][x])
    if to_root:
        x = top
        while x >= 0:
            if tree["left"][x] >= 0:
                nodes.add(x)
            x = int(tree["parent"][x])
    order = sorted(nodes, key=lambda p: -tree["depth"][p])
    return leaves, order, top


def algorithm2(store: HInv, series_frm, series_to, a: int, b: int, delta: float,
               to_root: bool = False) -> HInv:
    """Algorithm 2 on a copy of `store` (bus ids a, b in original order)."""
    t = store.tree
    new = copy.deepcopy(store)
    pa = int(t["pos"][a])
    pb = int(t["pos"][b]) if b >= 0 else -1
    if b >= 0:
        e = find_branch(series_frm, series_to, a, b)
        la, lb = leaf_of(t, pa), leaf_of(t, pb)
        if e < 0 and la != lb:
            raise ValueError("no branch between buses in different leaves")
        if e >= 0:
            new.g_branch = new.g_branch.copy()
            new.g_branch[e] += delta
    new.Gp = modified_G(store.Gp, pa, pb, delta)
    leaves, order, _ = touched_path(t, pa, pb, to_root)
    for j in leaves:
        new._build_node(j)
    for q in order:
        new._build_node(q)
    return new


def rebuild(store: HInv, series_frm, series_to, a: int, b: int, delta: float) -> HInv:
    """Explicit recomputation of the whole store on G' (Algorithm 1 again), the reference of
    Sec. IV's local modification."""
    t = store.tree
    G = np.empty_like(store.Gp)
    perm = t["perm"]
    G[np.ix_(perm, perm)] = store.Gp
    G2 = modified_G(G, a, b, delta)
    g = store.g_branch.copy()
    if b >= 0:
        e = find_branch(series_frm, series_to, a, b)
        if e >= 0:
            g[e] += delta
    return HInv(G2, t, g, store.mode)


def leaf_inversion_saving(d_th: int, n: int) -> float:
    """Share of matrix elements not re-inverted when only a d_th x d_th leaf is
    inverted instead of the n x n matrix (Sec. V-C.2): 1 - (d_th/n)^2."""
    return 1.0 - (d_th / n) ** 2
