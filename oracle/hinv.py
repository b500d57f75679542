"""Hierarchical inverse of G (oracle; test infrastructure).

Sec. III of the paper. For a node p with children l, r the conductance matrix
splits as G_p = [[G_l, H], [H^T, G_r]] (Eq. 3), and H = h_l h_r^T has rank k,
the number of branches cut between l and r (Sec. III-A, before Eq. 9). The
decomposition is not unique; the one used here gives one column per cut
branch e = (a in l, b in r):  h_l[:, e] = -g_e e_a,  h_r[:, e] = e_b,
so (h_l h_r^T)[a, b] = -g_e, the off-diagonal entry of G. Three-phase networks
partitioned by bus (partition.build_block_tree) take block cuts instead: one
column per (left bus, right node) pair of joined buses, h_l holding the three
entries G[x, y] of the left bus's nodes x and h_r = e_y, so a coupled line is a
rank-3 cut (b buses per leaf become 3b nodes).

Two stores share one shape. With P = Ginv_l h_l and Q = Ginv_r h_r (the
factors of Eq. 9) and Y = blkdiag(P, Q):

  PAPER  (Algorithm 1, Eq. 4 and 9): Ginv_p = [[Ginv_l, M], [M^T, Ginv_r]],
         M = -(Ginv_l h_l)(Ginv_r h_r)^T = -P Q^T, where Ginv_l, Ginv_r are
         the approximations of the children. Written as D^{-1} - Y C Y^T with
         the core C = [[0, I], [I, 0]].
  EXACT  G_p = D + W X W^T with D = blkdiag(G_l, G_r), W = blkdiag(h_l, h_r),
         X = [[0, I], [I, 0]] (X is its own inverse), so by the Woodbury
         identity G_p^{-1} = D^{-1} - Y S^{-1} Y^T with
         S = X + W^T D^{-1} W = [[h_l^T P, I], [I, h_r^T Q]]; the core is S^{-1}.
         This is the exact inverse whenever the children's are exact.

Leaves are inverted directly (Algorithm 1, "direct compute"); here by dense
Cholesky. Only leaf inverses, the factors P, Q and the cores are stored
(the storage claim at the end of Sec. III-B).
"""
from __future__ import annotations

import numpy as np

from . import dense as _dense

EXACT = 0
PAPER = 1


def _perm_matrix(G: np.ndarray, tree: dict) -> np.ndarray:
    """G in the nested ordering of the partition (Sec. III-B), so every node is a range."""
    p = tree["perm"]
    return G[np.ix_(p, p)]


class HInv:
    """The hierarchical store of Sec. III (Algorithm 1 for PAPER, Woodbury cores for EXACT; see
    the module header), over the tree in the nested ordering `tree['perm']`."""

    def __init__(self, G: np.ndarray, tree: dict, g_branch: np.ndarray, mode: int = EXACT):
        self.tree = tree
        self.mode = mode
        self.Gp = _perm_matrix(np.asarray(G, float), tree)   # G in nested order
        self.g_branch = np.asarray(g_branch, float)          # conductance per series branch id
        nn = len(tree["lo"])
        self.leaf_inv = {}
        self.P = {}
        self.Q = {}
        self.C = {}
        self.hl = {}
        self.hr = {}
        order = sorted(range(nn), key=lambda p: -tree["depth"][p])   # children before parents
        for p in order:
            self._build_node(p)

    # -- construction -----------------------------------------------------
    def node_range(self, p):
        """Positions [lo, hi) of node p in the nested ordering (Sec. III-B)."""
        return int(self.tree["lo"][p]), int(self.tree["hi"][p])

    def cut_columns(self, p):
        """h_l, h_r of node p (dense, n_l x k and n_r x k): H = h_l h_r^T of Eq. 3, one column per
    cut branch (Sec. III-A, before Eq. 9). Block trees (partition.build_block_tree, key cut_w = B)
    have B left entries per column, h_l[x, c] = G[x, y] for the B vertices x of the left group and
    h_r = e_y."""
        t = self.tree
        l, r = int(t["left"][p]), int(t["right"][p])
        ll, lh = self.node_range(l)
        rl, rh = self.node_range(r)
        s, e = int(t["cut_ptr"][p]), int(t["cut_ptr"][p + 1])
        k = e - s
        W = int(t.get("cut_w", 1))
        hl = np.zeros((lh - ll, k))
        hr = np.zeros((rh - rl, k))
        for c in range(k):
            b = int(t["cut_b"][s + c])
            if W == 1:
                a = int(t["cut_a"][s + c]); br = int(t["cut_e"][s + c])
                hl[a - ll, c] = -self.g_branch[br]
            else:
                for w in range(W):
                    a = int(t["cut_a"][W * (s + c) + w])
                    hl[a - ll, c] = self.Gp[a, b]
            hr[b - rl, c] = 1.0
        return hl, hr

    def _build_node(self, p):
        """Algorithm 1 at node p: a leaf's direct inverse, or P, Q of Eq. 9 from the children's
        stores and the node's core (PAPER: [[0, I], [I, 0]]; EXACT: S^{-1})."""
        t = self.tree
        lo, hi = self.node_range(p)
        if t["left"][p] < 0:
            self.leaf_inv[p] = _dense.inverse(self.Gp[lo:hi, lo:hi])
            return
        l, r = int(t["left"][p]), int(t["right"][p])
        hl, hr = self.cut_columns(p)
        self.hl[p], self.hr[p] = hl, hr
        P = self.apply_node(l, hl)
        Q = self.apply_node(r, hr)
        self.P[p], self.Q[p] = P, Q
        k = hl.shape[1]
        X = np.block([[np.zeros((k, k)), np.eye(k)], [np.eye(k), np.zeros((k, k))]])
        if self.mode == PAPER:
            self.C[p] = X
        else:
            S = X + np.block([[hl.T @ P, np.zeros((k, k))], [np.zeros((k, k)), hr.T @ Q]])
            self.C[p] = np.linalg.inv(S)

    # -- application --------------------------------------------------------
    def apply_node(self, p, X: np.ndarray) -> np.ndarray:
        """Ginv_p @ X by the recursive definition (Eq. 4 with Eq. 9's factors): children first,
        then the correction -Y C Y^T X of node p."""
        t = self.tree
        X = np.asarray(X, float)
        if t["left"][p] < 0:
            return self.leaf_inv[p] @ X
        l, r = int(t["left"][p]), int(t["right"][p])
        nl = int(t["hi"][l] - t["lo"][l])
        Xl, Xr = X[:nl], X[nl:]
        Yl = self.apply_node(l, Xl)
        Yr = self.apply_node(r, Xr)
        P, Q, C = self.P[p], self.Q[p], self.C[p]
        k = P.shape[1]
        tvec = np.concatenate([P.T @ Xl, Q.T @ Xr], axis=0)
        s = C @ tvec
        return np.concatenate([Yl - P @ s[:k], Yr - Q @ s[k:]], axis=0)

    def apply(self, x: np.ndarray) -> np.ndarray:
        """v = Ginv i (Eq. 2) with x, v in the original bus order."""
        perm = self.tree["perm"]
        x = np.asarray(x, float)
        y = self.apply_node(0, x[perm])
        out = np.empty_like(y)
        out[perm] = y
        return out

    def dense_node(self, p) -> np.ndarray:
        """Ginv_p as a dense matrix (applied to the identity), nested order."""
        lo, hi = self.node_range(p)
        return self.apply_node(p, np.eye(hi - lo))

    def dense(self) -> np.ndarray:
        """Ginv (Sec. III's approximation for PAPER, the exact inverse for EXACT) in the original
    bus order; Fig. 5 compares the two."""
        perm = self.tree["perm"]
        D = self.dense_node(0)
        out = np.empty_like(D)
        out[np.ix_(perm, perm)] = D
        return out


def algorithm1_dense(Gp: np.ndarray, tree: dict, p: int = 0) -> np.ndarray:
    """Algorithm 1 with dense blocks, straight from Eq. 4 and 7:
    Ginv_p = [[Ginv_l, M], [M^T, Ginv_r]], M = -Ginv_l H Ginv_r, H = G_lr.
    Gp is G in the nested ordering. An independent check of the factored
    PAPER store (it never forms h_l, h_r)."""
    lo, hi = int(tree["lo"][p]), int(tree["hi"][p])
    if tree["left"][p] < 0:
        return _dense.inverse(Gp[lo:hi, lo:hi])
    l, r = int(tree["left"][p]), int(tree["right"][p])
    A = algorithm1_dense(Gp, tree, l)
    B = algorithm1_dense(Gp, tree, r)
    ml = int(tree["hi"][l] - tree["lo"][l])
    H = Gp[lo:hi, lo:hi][:ml, ml:]
    M = -A @ H @ B
    return np.block([[A, M], [M.T, B]])


def relative_error(A: np.ndarray, B: np.ndarray) -> float:
    """||A - B||_F / ||B||_F, the reading of the paper's Fig. 5 error."""
    return float(np.linalg.norm(A - B) / np.linalg.norm(B))
