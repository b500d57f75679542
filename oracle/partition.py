"""Partition tree of the network (oracle; test infrastructure).

The paper recursively bisects the network into a binary tree whose leaves are
sub-networks of bounded size and asks the bisection to minimise the branches
between the two halves (Sec. III-B, Fig. 2-3); the algorithm itself is
delegated to the authors' earlier work and not given. The reading adopted
here is a deterministic, integer-only recursive bisection, written out
independently of the GPU library's C++ version so the two can be compared
array for array:

  1. Start vertex: BFS from the smallest bus id of the set; take the farthest
     reached vertex (ties -> smallest id); repeat once from there.
  2. Growth: BFS order from the start vertex (neighbours by ascending id; a
     fresh BFS from the smallest unvisited id when the set is disconnected).
     The first ceil(n/2) vertices form side A, the rest side B.
  3. Kernighan-Lin refinement, at most 4 passes. D(v) = external - internal
     branch count (parallel branches count separately). Each pass swaps
     floor(n/2) tentative pairs: a = argmax D over unlocked A, then
     b = argmax D(b) - 2 w(a,b) over unlocked B (ties -> smallest id),
     locks both and updates D as if swapped. The prefix with the largest
     cumulative gain (shortest on ties) is applied if its gain is > 0,
     otherwise refinement stops.
  4. The half holding the smaller minimum bus id is the left child.
  5. Splitting stops at depth `levels` (levels > 0), or when a set has at most
     d_th buses (levels == 0, leaf iff n <= d_th), or when n < 2.

Tree nodes are numbered breadth first (root 0). Leaves, read left to right,
define the nested ordering `perm` (buses ascending inside a leaf), so every
node is a contiguous range [lo, hi) of it. A node's cut list holds every
bus-to-bus branch with one end in each child, oriented (a in left, b in
right) and sorted by (position of a, position of b, branch id).
"""
from __future__ import annotations

from collections import deque

import numpy as np

_NEG = np.int64(-(1 << 60))


def _local_graph(V: np.ndarray, frm: np.ndarray, to: np.ndarray):
    """Induced subgraph on V (sorted global ids): neighbour lists (ascending,
    unique) and weights (branch multiplicities), the graph one bisection of
    Sec. III-B works on."""
    n = len(V)
    loc = {int(g): i for i, g in enumerate(V)}
    w = [dict() for _ in range(n)]
    for a, b in zip(frm, to):
        a = int(a); b = int(b)
        if b < 0 or a == b:
            continue
        ia = loc.get(a); ib = loc.get(b)
        if ia is None or ib is None:
            continue
        w[ia][ib] = w[ia].get(ib, 0) + 1
        w[ib][ia] = w[ib].get(ia, 0) + 1
    nbr = [np.array(sorted(d.keys()), dtype=np.int64) for d in w]
    wt = [np.array([d[k] for k in sorted(d.keys())], dtype=np.int64) for d in w]
    return nbr, wt


def _bfs(nbr, start, n):
    """Breadth-first distances and visit order from `start` (step 1 of the module header)."""
    dist = np.full(n, -1, np.int64)
    dist[start] = 0
    q = deque([start])
    order = []
    while q:
        u = q.popleft()
        order.append(u)
        for v in nbr[u]:
            if dist[v] < 0:
                dist[v] = dist[u] + 1
                q.append(int(v))
    return dist, order


def _start_vertex(nbr, n):
    """Step 1: the pseudo-peripheral start vertex (two BFS sweeps, ties to the smallest id)."""
    s = 0
    for _ in range(2):
        dist, _ = _bfs(nbr, s, n)
        m = dist.max()
        s = int(np.flatnonzero(dist == m)[0])
    return s


def _growth_order(nbr, start, n):
    """Step 2: BFS growth order from the start vertex, restarting at the smallest unvisited id."""
    seen = np.zeros(n, bool)
    order = []
    roots = [start] + list(range(n))
    for r in roots:
        if seen[r]:
            continue
        seen[r] = True
        q = deque([r])
        while q:
            u = q.popleft()
            order.append(u)
            for v in nbr[u]:
                if not seen[v]:
                    seen[v] = True
                    q.append(int(v))
    return order


def _kl(side: np.ndarray, nbr, wt, passes: int = 4) -> np.ndarray:
    """Step 3: Kernighan-Lin refinement of the two sides, minimising the cut branches that
    Sec. III-B asks the bisection to minimise."""
    n = len(side)
    side = side.copy()
    for _ in range(passes):
        D = np.zeros(n, np.int64)
        for v in range(n):
            if len(nbr[v]):
                ext = side[nbr[v]] != side[v]
                D[v] = int(wt[v][ext].sum()) - int(wt[v][~ext].sum())
        locked = np.zeros(n, bool)
        pairs, gains = [], []
        steps = min(int((side == 0).sum()), int((side == 1).sum()))
        for _s in range(steps):
            va = np.where((side == 0) & ~locked, D, _NEG)
            a = int(np.argmax(va))
            vb = np.where((side == 1) & ~locked, D, _NEG)
            wab = 0
            if len(nbr[a]):
                nb_a = nbr[a]
                inb = (side[nb_a] == 1) & ~locked[nb_a]
                vb[nb_a[inb]] -= 2 * wt[a][inb]
            b = int(np.argmax(vb))
            pos = np.searchsorted(nbr[a], b)
            if pos < len(nbr[a]) and nbr[a][pos] == b:
                wab = int(wt[a][pos])
            gains.append(int(D[a] + D[b] - 2 * wab))
            pairs.append((a, b))
            locked[a] = True
            locked[b] = True
            for x, wx in zip(nbr[a], wt[a]):
                if not locked[x]:
                    D[x] += 2 * wx if side[x] == 0 else -2 * wx
            for y, wy in zip(nbr[b], wt[b]):
                if not locked[y]:
                    D[y] += 2 * wy if side[y] == 1 else -2 * wy
        if not gains:
            break
        cum = np.cumsum(np.array(gains, np.int64))
        m = int(np.argmax(cum))
        if cum[m] <= 0:
            break
        for a, b in pairs[:m + 1]:
            side[a] = 1
            side[b] = 0
    return side


def bisect(V: np.ndarray, frm: np.ndarray, to: np.ndarray):
    """One bisection of Sec. III-B (steps 1-4 of the module header): split the sorted global id
    set V into (left, right), both sorted."""
    n = len(V)
    nbr, wt = _local_graph(V, frm, to)
    start = _start_vertex(nbr, n)
    order = _growth_order(nbr, start, n)
    nA = (n + 1) // 2
    side = np.ones(n, np.int64)
    side[np.array(order[:nA], np.int64)] = 0
    side = _kl(side, nbr, wt)
    A = V[side == 0]
    B = V[side == 1]
    if A.min() < B.min():
        return A, B
    return B, A


def cut_size(V_left, V_right, frm, to) -> int:
    """Branches between the two halves: the quantity a bisection minimises (Sec. III-B) and the
    rank k of H (Sec. III-A)."""
    L = set(int(x) for x in V_left)
    R = set(int(x) for x in V_right)
    c = 0
    for a, b in zip(frm, to):
        a = int(a); b = int(b)
        if b < 0:
            continue
        if (a in L and b in R) or (a in R and b in L):
            c += 1
    return c


def build_tree(n_bus: int, frm: np.ndarray, to: np.ndarray, levels: int = 0, d_th: int = 0) -> dict:
    """The partition tree of Sec. III-B (Fig. 2-3) by recursive bisection, with step 5's stopping
    rule. `frm/to` are the bus-to-bus branches (series branch ids are their positions in these
    arrays; to < 0 entries are ignored)."""
    frm = np.asarray(frm, np.int64)
    to = np.asarray(to, np.int64)
    buses = [np.arange(n_bus, dtype=np.int64)]
    depth = [0]
    parent = [-1]
    left = [-1]
    right = [-1]
    i = 0
    while i < len(buses):
        V = buses[i]
        n = len(V)
        split = n >= 2 and ((levels > 0 and depth[i] < levels) or (levels <= 0 and n > d_th))
        if split:
            A, B = bisect(V, frm, to)
            for part in (A, B):
                buses.append(part)
                depth.append(depth[i] + 1)
                parent.append(i)
                left.append(-1)
                right.append(-1)
            left[i] = len(buses) - 2
            right[i] = len(buses) - 1
        i += 1
    nn = len(buses)
    lo = np.zeros(nn, np.int64)
    hi = np.zeros(nn, np.int64)
    perm = []
    leaves = []

    def dfs(p):
        # leaves left to right give the nested ordering; every node becomes a range
        lo[p] = len(perm)
        if left[p] < 0:
            perm.extend(int(x) for x in buses[p])
            leaves.append(p)
        else:
            dfs(left[p])
            dfs(right[p])
        hi[p] = len(perm)

    dfs(0)
    perm = np.array(perm, np.int64)
    pos = np.empty(n_bus, np.int64)
    pos[perm] = np.arange(n_bus)
    cut_ptr = [0]
    cut_a, cut_b, cut_e = [], [], []
    for p in range(nn):
        if left[p] >= 0:
            l, r = left[p], right[p]
            rows = []
            for e, (a, b) in enumerate(zip(frm, to)):
                if b < 0:
                    continue
                pa, pb = pos[a], pos[b]
                if lo[l] <= pa < hi[l] and lo[r] <= pb < hi[r]:
                    rows.append((int(pa), int(pb), e))
                elif lo[l] <= pb < hi[l] and lo[r] <= pa < hi[r]:
                    rows.append((int(pb), int(pa), e))
            rows.sort()
            for pa, pb, e in rows:
                cut_a.append(pa); cut_b.append(pb); cut_e.append(e)
        cut_ptr.append(len(cut_a))
    return dict(n_bus=n_bus, perm=perm, pos=pos, lo=lo, hi=hi,
                parent=np.array(parent, np.int64), left=np.array(left, np.int64),
                right=np.array(right, np.int64), depth=np.array(depth, np.int64),
                leaves=np.array(leaves, np.int64),
                cut_ptr=np.array(cut_ptr, np.int64), cut_a=np.array(cut_a, np.int64),
                cut_b=np.array(cut_b, np.int64), cut_e=np.array(cut_e, np.int64))


def build_block_tree(n_node: int, frm: np.ndarray, to: np.ndarray, B: int, levels: int = 0,
                     d_th: int = 0) -> dict:
    """Partition tree whose units are groups of B consecutive vertices (the three nodes of a
    three-phase bus, so that a leaf of b buses holds 3b nodes), with block cuts.

    The paper counts three nodes per bus (Sec. III-A, after Eq. 3) and bisects buses (Sec. III-B).
    Here the group graph has one edge per distinct pair of groups joined by any vertex branch
    (x // B != y // B, y >= 0), listed as (min, max) in ascending order; build_tree bisects it
    (d_th counts vertices: a group leaf holds at most d_th // B groups). Positions expand group
    by group: vertex B g + w sits at B pos_g[g] + w.

    A node's cut columns factor the off-diagonal block of Eq. 3 exactly, H = G_lr = h_l h_r^T,
    with one column per (left group A, right vertex y) pair whose groups are joined:
    h_r = e_y and h_l holds G[x, y] at the B vertices x of A. A coupled three-phase line is then
    one rank-3 cut (B columns) instead of one column per vertex branch. Columns are sorted by
    (position of A's first vertex, position of y); cut_a holds B positions per column
    (cut_a[B c + w]), cut_e is -1 (the coefficients come from G itself)."""
    frm = np.asarray(frm, np.int64)
    to = np.asarray(to, np.int64)
    if B < 1 or n_node % B:
        raise ValueError("n_node must be a multiple of B")
    ng = n_node // B
    pairs = sorted({(min(int(x) // B, int(y) // B), max(int(x) // B, int(y) // B))
                    for x, y in zip(frm, to) if y >= 0 and int(x) // B != int(y) // B})
    gf = np.array([a for a, _ in pairs], np.int64)
    gt = np.array([b for _, b in pairs], np.int64)
    tg = build_tree(ng, gf, gt, levels=levels, d_th=d_th // B if levels <= 0 else 0)
    nn = len(tg["lo"])
    perm = (B * tg["perm"][:, None] + np.arange(B)[None, :]).reshape(-1)
    pos = np.empty(n_node, np.int64)
    pos[perm] = np.arange(n_node)
    lo, hi = B * tg["lo"], B * tg["hi"]
    gpos = tg["pos"]
    cut_ptr = [0]
    cut_a, cut_b = [], []
    for p in range(nn):
        l, r = int(tg["left"][p]), int(tg["right"][p])
        if l >= 0:
            cols = []
            for a, b in pairs:
                pa, pb = int(gpos[a]), int(gpos[b])
                if tg["lo"][l] <= pa < tg["hi"][l] and tg["lo"][r] <= pb < tg["hi"][r]:
                    A, Bb = pa, pb
                elif tg["lo"][l] <= pb < tg["hi"][l] and tg["lo"][r] <= pa < tg["hi"][r]:
                    A, Bb = pb, pa
                else:
                    continue
                for q in range(B):
                    cols.append((B * A, B * Bb + q))
            cols.sort()
            for a0, y in cols:
                cut_a.extend(a0 + w for w in range(B))
                cut_b.append(y)
        cut_ptr.append(len(cut_b))
    return dict(n_bus=n_node, perm=perm, pos=pos, lo=lo, hi=hi, parent=tg["parent"], left=tg["left"],
                right=tg["right"], depth=tg["depth"], leaves=tg["leaves"],
                cut_ptr=np.array(cut_ptr, np.int64), cut_a=np.array(cut_a, np.int64),
                cut_b=np.array(cut_b, np.int64), cut_e=np.full(len(cut_b), -1, np.int64), cut_w=B)


def leaf_of(tree: dict, position: int) -> int:
    """The leaf holding a position: where Algorithm 2 starts (Sec. IV)."""
    for j in tree["leaves"]:
        if tree["lo"][j] <= position < tree["hi"][j]:
            return int(j)
    raise ValueError(position)


def lca(tree: dict, u: int, v: int) -> int:
    """Lowest common ancestor of two tree nodes by walking parent pointers (the LCA that
    Algorithm 2 updates up to, Sec. IV)."""
    anc = set()
    x = u
    while x >= 0:
        anc.add(x)
        x = int(tree["parent"][x])
    x = v
    while x not in anc:
        x = int(tree["parent"][x])
    return x
