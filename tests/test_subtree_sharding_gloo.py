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

The second test runs whole time steps this way (injection, sharded apply, history update of the
rank's elements). A branch joining two ranks' subtrees is cut at a top node, so both its end
voltages follow from the values that one all-gather already brings: one exchange per step
suffices for the whole time loop.
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


def _rank_steps(rank, world, port, q, n_steps):
    import torch.distributed as dist
    from oracle import companion as cm
    from oracle import emt as oemt
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nw, H = _store()
        t, net, el = H.tree, nw.net, nw.el
        n = nw.G.shape[0]
        perm = np.asarray(t["perm"])
        pos = np.empty(n, np.int64)
        pos[perm] = np.arange(n)
        d = int(np.log2(world))
        owned = sorted((p for p in range(len(t["lo"])) if t["depth"][p] == d), key=lambda p: t["lo"][p])
        me = owned[rank]
        lo, hi = int(t["lo"][me]), int(t["hi"][me])
        top = [p for p in range(len(t["lo"])) if t["depth"][p] < d and t["left"][p] >= 0]
        ends = sorted({int(v) for p in top for c in range(t["cut_ptr"][p], t["cut_ptr"][p + 1])
                       for v in (t["cut_a"][c], t["cut_b"][c])})
        subtree_of = {}
        for o in owned:
            for x in range(int(t["lo"][o]), int(t["hi"][o])):
                subtree_of[x] = o

        def top_anc(x, below_depth):
            out, p = [], int(t["parent"][subtree_of[x]])
            while p >= 0:
                if t["depth"][p] > below_depth:
                    out.append(p)
                p = int(t["parent"][p])
            return out

        # the rank's elements: every element with an end in its range; a cross-rank element is a
        # top-node cut branch, so its far end is a gathered endpoint
        ea, eb = pos[el["a"]], np.where(el["b"] >= 0, pos[np.maximum(el["b"], 0)], -1)
        mine_el = ((ea >= lo) & (ea < hi)) | ((eb >= lo) & (eb < hi))
        far = sorted({int(x) for x in np.concatenate([ea[mine_el], eb[mine_el]]) if x >= 0 and not lo <= x < hi})
        assert set(far) <= set(ends)
        Ih = np.zeros(len(el["g"]))
        active = np.ones(len(el["g"]), bool)
        rec = np.zeros((n_steps, hi - lo))
        for step in range(1, n_steps + 1):
            rhs = cm.source_injection(net, step * DT) + cm.history_injection(el, np.where(mine_el, Ih, 0.0), n)
            Y = H.apply_node(me, rhs[perm][lo:hi])
            gathered = [None] * world
            dist.all_gather_object(gathered, {e: float(Y[e - lo]) for e in ends if lo <= e < hi})
            yend = {}
            for part in gathered:
                yend.update(part)
            s = {}

            def value_below(x, depth):
                # the solve of the subtree below depth `depth` at position x (-1: the whole network)
                v = yend[x]
                for a in top_anc(x, depth):
                    row, half = _top_rows(H, a, x)
                    v -= row @ s[a][half]
                return v

            for p in sorted(top, key=lambda p: -t["depth"][p]):
                c0, c1 = int(t["cut_ptr"][p]), int(t["cut_ptr"][p + 1])
                tl = [-H.g_branch[t["cut_e"][c]] * value_below(int(t["cut_a"][c]), t["depth"][p])
                      for c in range(c0, c1)]
                tr = [value_below(int(t["cut_b"][c]), t["depth"][p]) for c in range(c0, c1)]
                s[p] = H.C[p] @ np.array(tl + tr)
            v = Y.copy()
            for i in range(hi - lo):
                for a in top_anc(lo + i, -1):
                    row, half = _top_rows(H, a, lo + i)
                    v[i] -= row @ s[a][half]
            vb = np.full(n, np.nan)   # bus voltages this rank knows: its own and the far ends
            vb[perm[lo:hi]] = v
            for x in far:
                vb[perm[x]] = value_below(x, -1)
            with np.errstate(invalid="ignore"):
                _, Ih_new = cm.update_history(el, vb, Ih, active)
            Ih = np.where(mine_el, Ih_new, Ih)
            assert np.all(np.isfinite(Ih[mine_el]))
            rec[step - 1] = v
        ref, _ = oemt.simulate(nw, n_steps, (), solver="exact")
        want = ref[:, perm[lo:hi]]
        q.put((rank, float(np.max(np.abs(rec - want)) / np.max(np.abs(want))), len(far), len(ends)))
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


@pytest.mark.parametrize("world", [2, 4])
def test_subtree_sharded_time_steps_equal_whole_network(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    n_steps = 40
    procs = [ctx.Process(target=_rank_steps, args=(r, world, port, q, n_steps)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, err, n_far, n_ends in out:
        assert not isinstance(err, str), (rank, err)
        assert err <= 1e-11, (rank, err)
        assert 0 < n_far <= n_ends   # cross-rank elements exist, and their far ends are gathered anyway
