"""One network sharded by subtree over CPU ranks (gloo): the data flow of a multi-GPU apply.

Rank r of 2^d owns the r-th subtree at depth d (its leaves, and its rows of every factor). One
apply v = G^-1 i is then: (1) each rank solves its own subtree, Y_r = G_sub^-1 i_sub; (2) one
exchange, an all-gather of each rank's Y_r at the cut endpoints of the top nodes (depth < d),
a few hundred values; (3) every rank runs the boundary sweep of the top nodes redundantly, from
the gathered values and the factor rows at those endpoints (replicated): the child's solve at an
endpoint is Y minus the corrections of the top nodes below, t_p = [h_l^T y_l; h_r^T y_r] and
s_p = C_p t_p (Eq. 9 factors, exact cores); (4) each rank expands its own rows,
v = Y_r - sum over its top ancestors of F row . s(half). The assembled result must equal the
hierarchical apply of the whole network. No GPU is used: the store and the per-rank arithmetic are
the oracle's.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

DT = 50e-6


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _store():
    import netgen
    from oracle import emt as oemt, hinv as ohinv
    nw = oemt.Network(netgen.tiled(2, 4), DT, levels=3)
    return nw, ohinv.HInv(nw.G, nw.tree, nw.g_series, ohinv.EXACT)


def _top_rows(H, p, x):
    # factor row of top node p at position x and the half of s it multiplies
    t = H.tree
    l, r = int(t["left"][p]), int(t["right"][p])
    k = H.P[p].shape[1]
    if x < t["hi"][l]:
        return H.P[p][x - t["lo"][l]], slice(0, k)
    return H.Q[p][x - t["lo"][r]], slice(k, 2 * k)


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nw, H = _store()
        t = H.tree
        d = int(np.log2(world))
        x = np.random.default_rng(31).standard_normal(nw.G.shape[0])[t["perm"]]   # right-hand side, nested order
        owned = sorted((p for p in range(len(t["lo"])) if t["depth"][p] == d), key=lambda p: t["lo"][p])
        me = owned[rank]
        lo, hi = int(t["lo"][me]), int(t["hi"][me])
        # (1) own subtree solve
        Y = H.apply_node(me, x[lo:hi])
        # (2) one exchange: own values at the cut endpoints of the top nodes
        top = [p for p in range(len(t["lo"])) if t["depth"][p] < d and t["left"][p] >= 0]
        ends = sorted({int(v) for p in top for c in range(t["cut_ptr"][p], t["cut_ptr"][p + 1])
                       for v in (t["cut_a"][c], t["cut_b"][c])})
        mine = {e: float(Y[e - lo]) for e in ends if lo <= e < hi}
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        yend = {}
        for part in gathered:
            yend.update(part)
        # (3) top sweep, bottom-up, redundantly on every rank
        s = {}

        def anc_top(pos, below_depth):
            # top ancestors of a position with depth > below_depth, deepest first
            out = []
            p = int(t["parent"][owned[[t["lo"][o] <= pos < t["hi"][o] for o in owned].index(True)]])
            while p >= 0:
                if t["depth"][p] > below_depth:
                    out.append(p)
                p = int(t["parent"][p])
            return out

        def child_value(pos, p):
            v = yend[pos]
            for a in anc_top(pos, t["depth"][p]):
                row, half = _top_rows(H, a, pos)
                v -= row @ s[a][half]
            return v

        for p in sorted(top, key=lambda p: -t["depth"][p]):
            c0, c1 = int(t["cut_ptr"][p]), int(t["cut_ptr"][p + 1])
            tl = [-H.g_branch[t["cut_e"][c]] * child_value(int(t["cut_a"][c]), p) for c in range(c0, c1)]
            tr = [child_value(int(t["cut_b"][c]), p) for c in range(c0, c1)]
            s[p] = H.C[p] @ np.array(tl + tr)
        # (4) local expansion of the own rows
        v = Y.copy()
        for i in range(hi - lo):
            for a in anc_top(lo + i, -1):
                row, half = _top_rows(H, a, lo + i)
                v[i] -= row @ s[a][half]
        ref = H.apply_node(0, x)[lo:hi]
        q.put((rank, float(np.max(np.abs(v - ref)) / np.max(np.abs(ref))), len(mine), len(ends)))
    except Exception as e:   # report instead of leaving the parent waiting
        q.put((rank, repr(e), -1, -1))
        raise
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_subtree_sharded_apply_equals_whole_apply(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n_bus = 1432
    for rank, err, n_mine, n_ends in out:
        assert not isinstance(err, str), (rank, err)
        assert err <= 1e-12, (rank, err)
        assert n_ends < 0.05 * n_bus   # the single exchange: a few hundred values, not a vector
    assert sum(o[2] for o in out) == out[0][3]   # every endpoint comes from exactly one rank
