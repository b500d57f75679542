// Partition tree: deterministic recursive bisection (Sec. III-B, Fig. 2-3).
//
// The paper asks the bisection to minimise the branches between the halves and delegates the
// algorithm to earlier work. This implementation fixes one deterministic, integer-only reading:
//   1. start vertex: BFS from the smallest bus id of the set, take the farthest vertex (ties ->
//      smallest id), BFS again from it and take the farthest again;
//   2. growth: BFS order from the start (neighbours by ascending id, a fresh BFS from the
//      smallest unvisited id when the set is disconnected); the first ceil(n/2) form side A;
//   3. Kernighan-Lin refinement, at most 4 passes, gains in branch counts: per pass floor(n/2)
//      tentative swaps, a = argmax D over unlocked A, b = argmax D(b) - 2 w(a,b) over unlocked
//      B, smallest id on ties; the best prefix is applied if its gain is positive;
//   4. the half with the smaller minimum bus id becomes the left child;
//   5. leaves at depth `levels`, or (levels == 0) once a set has at most d_th buses.
// Nodes are numbered breadth first; the left-to-right leaves give the nested ordering.
#include <algorithm>
#include <cstdint>
#include <atomic>
#include <exception>
#include <mutex>
#include <thread>
#include <tuple>

#include "internal.h"

namespace emt {
namespace {

struct Local {
  int n = 0;
  std::vector<int> ptr;   // [n + 1]: vertex v's neighbours are adj[ptr[v] .. ptr[v + 1])
  std::vector<int> adj;   // ascending unique neighbours
  std::vector<int> wt;    // their multiplicities
};

// Induced subgraph on the set V (owner[v] == set, loc[v] its local index): ascending unique
// neighbours with their multiplicities.
Local local_graph(const std::vector<int>& V, int set, const std::vector<int>& owner, const std::vector<int>& loc,
                  const std::vector<std::vector<int>>& adj_global) {
  Local g;
  g.n = (int)V.size();
  g.ptr.assign(g.n + 1, 0);
  std::vector<int> tmp;
  for (int i = 0; i < g.n; ++i) {
    tmp.clear();
    for (int u : adj_global[V[i]])
      if (owner[u] == set && loc[u] != i) tmp.push_back(loc[u]);
    std::sort(tmp.begin(), tmp.end());
    for (size_t k = 0; k < tmp.size();) {
      size_t e = k;
      while (e < tmp.size() && tmp[e] == tmp[k]) ++e;
      g.adj.push_back(tmp[k]);
      g.wt.push_back((int)(e - k));
      k = e;
    }
    g.ptr[i + 1] = (int)g.adj.size();
  }
  return g;
}

std::vector<int> bfs_dist(const Local& g, int s) {
  std::vector<int> d(g.n, -1), q(g.n);
  int head = 0, tail = 0;
  d[s] = 0;
  q[tail++] = s;
  while (head < tail) {
    const int u = q[head++];
    for (int k = g.ptr[u]; k < g.ptr[u + 1]; ++k) {
      const int v = g.adj[k];
      if (d[v] < 0) {
        d[v] = d[u] + 1;
        q[tail++] = v;
      }
    }
  }
  return d;
}

int start_vertex(const Local& g) {
  int s = 0;
  for (int r = 0; r < 2; ++r) {
    std::vector<int> d = bfs_dist(g, s);
    int best = 0;
    for (int i = 1; i < g.n; ++i)
      if (d[i] > d[best]) best = i;
    s = best;
  }
  return s;
}

std::vector<int> growth_order(const Local& g, int start) {
  std::vector<char> seen(g.n, 0);
  std::vector<int> order;   // doubles as the BFS queue: a vertex is appended when first seen
  order.reserve(g.n);
  auto run = [&](int r) {
    if (seen[r]) return;
    seen[r] = 1;
    size_t head = order.size();
    order.push_back(r);
    while (head < order.size()) {
      const int u = order[head++];
      for (int k = g.ptr[u]; k < g.ptr[u + 1]; ++k) {
        const int v = g.adj[k];
        if (!seen[v]) {
          seen[v] = 1;
          order.push_back(v);
        }
      }
    }
  };
  run(start);
  for (int r = 0; r < g.n; ++r) run(r);
  return order;
}

// Unlocked vertices of one side bucketed by gain D (Fiduccia-Mattheyses style): per gain value a
// two-level bitset over vertex ids, so the argmax of (D[v], -v) is the lowest id of the highest
// non-empty bucket, and the next candidates in that order follow with a few word scans. Gains are
// branch counts, |D| <= the vertex's weighted degree.
struct GainBuckets {
  int W = 0, S = 0, off = 0, nb = 0;
  std::vector<uint64_t> b1, b2;   // [nb][W] vertex bits, [nb][S] non-empty words of b1
  std::vector<int> cnt;           // vertices per bucket
  int top = -1;                   // no bucket above is non-empty
  void init(int n, int max_abs) {
    W = (n + 63) / 64;
    S = (W + 63) / 64;
    off = max_abs;
    nb = 2 * max_abs + 1;
    b1.assign((size_t)nb * W, 0);
    b2.assign((size_t)nb * S, 0);
    cnt.assign(nb, 0);
    top = -1;
  }
  void insert(int v, int d) {
    const int k = d + off;
    uint64_t& w = b1[(size_t)k * W + (v >> 6)];
    if (!w) b2[(size_t)k * S + (v >> 12)] |= 1ull << ((v >> 6) & 63);
    w |= 1ull << (v & 63);
    ++cnt[k];
    top = std::max(top, k);
  }
  void erase(int v, int d) {
    const int k = d + off;
    uint64_t& w = b1[(size_t)k * W + (v >> 6)];
    w &= ~(1ull << (v & 63));
    if (!w) b2[(size_t)k * S + (v >> 12)] &= ~(1ull << ((v >> 6) & 63));
    --cnt[k];
  }
  // lowest id >= v in bucket k, or -1
  int next(int k, int v) const {
    const uint64_t* w1 = &b1[(size_t)k * W];
    const uint64_t* w2 = &b2[(size_t)k * S];
    int wi = v >> 6;
    if (wi >= W) return -1;
    const uint64_t m = w1[wi] & (~0ull << (v & 63));
    if (m) return (wi << 6) + __builtin_ctzll(m);
    int si = (wi + 1) >> 6;
    if (si >= S) return -1;
    uint64_t sm = ((wi + 1) & 63) ? (w2[si] & (~0ull << ((wi + 1) & 63))) : w2[si];
    while (true) {
      if (sm) {
        const int wj = (si << 6) + __builtin_ctzll(sm);
        return (wj << 6) + __builtin_ctzll(w1[wj]);
      }
      if (++si >= S) return -1;
      sm = w2[si];
    }
  }
  // argmax of (D, -id) over the bucketed vertices for which skip(v) is false; -1 if none
  template <class F>
  int best(F skip) {
    while (top >= 0 && cnt[top] == 0) --top;
    for (int k = top; k >= 0; --k) {
      if (!cnt[k]) continue;
      for (int v = next(k, 0); v >= 0; v = next(k, v + 1))
        if (!skip(v)) return v;
    }
    return -1;
  }
};

// The choices are those of the plain O(n) scans (a = largest D over unlocked A, b = largest
// D(b) - 2 w(a, b) over unlocked B, smallest id on ties): each side's unlocked vertices sit in
// gain buckets; for b the only values that differ from D are those of a's neighbours, so b is the
// better of the best neighbour and the best non-neighbour of the buckets.
void kernighan_lin(const Local& g, std::vector<int>& side, int passes) {
  const int n = g.n;
  std::vector<int> D(n), nbr_of(n, -1);   // nbr_of[u] == a: u is a neighbour of the current a
  std::vector<char> locked(n);
  int max_abs = 0;
  for (int v = 0; v < n; ++v) {
    int s = 0;
    for (int k = g.ptr[v]; k < g.ptr[v + 1]; ++k) s += g.wt[k];
    max_abs = std::max(max_abs, s);
  }
  GainBuckets T[2];
  for (int pass = 0; pass < passes; ++pass) {
    int nA = 0;
    for (int v = 0; v < n; ++v) {
      int s = 0;
      for (int k = g.ptr[v]; k < g.ptr[v + 1]; ++k) s += (side[g.adj[k]] != side[v]) ? g.wt[k] : -g.wt[k];
      D[v] = s;
      nA += side[v] == 0;
    }
    std::fill(locked.begin(), locked.end(), 0);
    T[0].init(n, max_abs);
    T[1].init(n, max_abs);
    for (int v = 0; v < n; ++v) T[side[v]].insert(v, D[v]);
    const int steps = std::min(nA, n - nA);
    std::vector<std::pair<int, int>> pairs;
    std::vector<long long> gains;
    pairs.reserve(steps);
    gains.reserve(steps);
    for (int st = 0; st < steps; ++st) {
      const int a = T[0].best([](int) { return false; });
      const int* na = g.adj.data() + g.ptr[a];
      const int* wa = g.wt.data() + g.ptr[a];
      const int da = g.ptr[a + 1] - g.ptr[a];
      // best neighbour of a in unlocked B, by D - 2 w
      bool have = false;
      long long bv = 0;
      int b = -1;
      long long wab = 0;
      for (int k = 0; k < da; ++k) {
        const int u = na[k];
        nbr_of[u] = a;
        if (side[u] != 1 || locked[u]) continue;
        const long long val = (long long)D[u] - 2LL * wa[k];
        if (!have || val > bv || (val == bv && u < b)) {
          have = true;
          bv = val;
          b = u;
          wab = wa[k];
        }
      }
      // best unlocked B vertex that is not a neighbour of a
      const int c = T[1].best([&](int v) { return nbr_of[v] == a; });
      if (c >= 0) {
        const long long val = D[c];
        if (!have || val > bv || (val == bv && c < b)) {
          have = true;
          bv = val;
          b = c;
          wab = 0;
        }
      }
      gains.push_back((long long)D[a] + D[b] - 2 * wab);
      pairs.emplace_back(a, b);
      locked[a] = 1;
      locked[b] = 1;
      T[0].erase(a, D[a]);
      T[1].erase(b, D[b]);
      for (int k = 0; k < da; ++k) {
        const int x = na[k];
        if (locked[x]) continue;
        T[side[x]].erase(x, D[x]);
        D[x] += (side[x] == 0) ? 2 * wa[k] : -2 * wa[k];
        T[side[x]].insert(x, D[x]);
      }
      for (int k = g.ptr[b]; k < g.ptr[b + 1]; ++k) {
        const int y = g.adj[k];
        if (locked[y]) continue;
        T[side[y]].erase(y, D[y]);
        D[y] += (side[y] == 1) ? 2 * g.wt[k] : -2 * g.wt[k];
        T[side[y]].insert(y, D[y]);
      }
    }
    if (gains.empty()) break;
    long long cum = 0, bestcum = 0;
    int m = -1;
    for (size_t i = 0; i < gains.size(); ++i) {
      cum += gains[i];
      if (m < 0 || cum > bestcum) { bestcum = cum; m = (int)i; }
    }
    if (bestcum <= 0) break;
    for (int i = 0; i <= m; ++i) {
      side[pairs[i].first] = 1;
      side[pairs[i].second] = 0;
    }
  }
}

}  // namespace

Tree build_tree(int n_bus, int n_branch, const int32_t* from, const int32_t* to, int levels,
                int d_th) {
  EMT_REQUIRE(n_bus >= 1, EMT_ERR_INVALID, "n_bus must be >= 1");
  EMT_REQUIRE(levels > 0 || d_th >= 1, EMT_ERR_INVALID, "need levels > 0 or d_th >= 1");
  std::vector<std::vector<int>> adj(n_bus);
  for (int e = 0; e < n_branch; ++e) {
    int a = from[e], b = to[e];
    EMT_REQUIRE(a >= 0 && a < n_bus && b >= -1 && b < n_bus, EMT_ERR_INVALID, "branch endpoint out of range");
    if (b < 0 || a == b) continue;
    adj[a].push_back(b);
    adj[b].push_back(a);
  }
  std::vector<std::vector<int>> sets;
  std::vector<int> depth, parent, left, right;
  sets.emplace_back(n_bus);
  for (int i = 0; i < n_bus; ++i) sets[0][i] = i;
  depth.push_back(0);
  parent.push_back(-1);
  left.push_back(-1);
  right.push_back(-1);
  // Level by level: the sets of one depth are disjoint, so their bisections run concurrently (each
  // is deterministic), and their children are appended in the parents' order, which keeps the
  // breadth-first numbering of a one-at-a-time loop.
  std::vector<int> owner(n_bus, -1), loc(n_bus, -1);
  size_t lvl_begin = 0;
  while (lvl_begin < sets.size()) {
    const size_t lvl_end = sets.size();
    std::vector<size_t> todo;
    for (size_t i = lvl_begin; i < lvl_end; ++i) {
      const int n = (int)sets[i].size();
      if (n >= 2 && ((levels > 0 && depth[i] < levels) || (levels <= 0 && n > d_th))) todo.push_back(i);
    }
    // owner[v] = index in `todo` of the set v belongs to at this depth, -1 for a vertex of a set
    // that is not bisected here (a leaf already): an index left from an earlier depth would make
    // it look like a member of whichever set now has that index
    std::fill(owner.begin(), owner.end(), -1);
    for (size_t q = 0; q < todo.size(); ++q) {
      const std::vector<int>& V = sets[todo[q]];
      for (int k = 0; k < (int)V.size(); ++k) {
        owner[V[k]] = (int)q;
        loc[V[k]] = k;
      }
    }
    std::vector<std::pair<std::vector<int>, std::vector<int>>> halves(todo.size());
    auto bisect = [&](size_t q) {
      const std::vector<int>& V = sets[todo[q]];
      const int n = (int)V.size();
      Local g = local_graph(V, (int)q, owner, loc, adj);
      const int s = start_vertex(g);
      std::vector<int> order = growth_order(g, s);
      std::vector<int> side(n, 1);
      const int nA = (n + 1) / 2;
      for (int k = 0; k < nA; ++k) side[order[k]] = 0;
      kernighan_lin(g, side, 4);
      std::vector<int> A, B;
      for (int k = 0; k < n; ++k) (side[k] == 0 ? A : B).push_back(V[k]);
      if (!(A.front() < B.front())) std::swap(A, B);
      halves[q] = {std::move(A), std::move(B)};
    };
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const size_t nth = std::min<size_t>(todo.size(), hw);
    if (nth <= 1) {
      for (size_t q = 0; q < todo.size(); ++q) bisect(q);
    } else {
      std::atomic<size_t> next{0};
      std::vector<std::thread> pool;
      std::exception_ptr err;
      std::mutex err_mu;
      for (size_t w = 0; w < nth; ++w)
        pool.emplace_back([&] {
          for (size_t q; (q = next.fetch_add(1)) < todo.size();) {
            try {
              bisect(q);
            } catch (...) {
              std::lock_guard<std::mutex> lk(err_mu);
              if (!err) err = std::current_exception();
            }
          }
        });
      for (auto& th : pool) th.join();
      if (err) std::rethrow_exception(err);
    }
    for (size_t q = 0; q < todo.size(); ++q) {
      const size_t i = todo[q];
      const int li = (int)sets.size();
      sets.push_back(std::move(halves[q].first));
      sets.push_back(std::move(halves[q].second));
      for (int c = 0; c < 2; ++c) {
        depth.push_back(depth[i] + 1);
        parent.push_back((int)i);
        left.push_back(-1);
        right.push_back(-1);
      }
      left[i] = li;
      right[i] = li + 1;
    }
    lvl_begin = lvl_end;
  }
  Tree t;
  t.n_bus = n_bus;
  const int nn = (int)sets.size();
  t.lo.assign(nn, 0);
  t.hi.assign(nn, 0);
  t.parent = parent;
  t.left = left;
  t.right = right;
  t.depth = depth;
  t.max_depth = *std::max_element(depth.begin(), depth.end());
  // nested ordering by a left-to-right walk (explicit stack, no recursion depth limit)
  std::vector<std::pair<int, int>> stack{{0, 0}};
  while (!stack.empty()) {
    auto [p, stage] = stack.back();
    stack.pop_back();
    if (stage == 0) {
      t.lo[p] = (int)t.perm.size();
      if (left[p] < 0) {
        for (int b : sets[p]) t.perm.push_back(b);
        t.leaves.push_back(p);
        t.hi[p] = (int)t.perm.size();
      } else {
        stack.push_back({p, 1});
        stack.push_back({right[p], 0});
        stack.push_back({left[p], 0});
      }
    } else {
      t.hi[p] = (int)t.perm.size();
    }
  }
  t.pos.assign(n_bus, 0);
  for (int i = 0; i < n_bus; ++i) t.pos[t.perm[i]] = i;
  t.cut_ptr.push_back(0);
  for (int p = 0; p < nn; ++p) {
    if (left[p] >= 0) {
      int l = left[p], r = right[p];
      std::vector<std::tuple<int, int, int>> rows;
      for (int e = 0; e < n_branch; ++e) {
        int a = from[e], b = to[e];
        if (b < 0) continue;
        int pa = t.pos[a], pb = t.pos[b];
        if (t.lo[l] <= pa && pa < t.hi[l] && t.lo[r] <= pb && pb < t.hi[r])
          rows.emplace_back(pa, pb, e);
        else if (t.lo[l] <= pb && pb < t.hi[l] && t.lo[r] <= pa && pa < t.hi[r])
          rows.emplace_back(pb, pa, e);
      }
      std::sort(rows.begin(), rows.end());
      for (auto& r3 : rows) {
        t.cut_a.push_back(std::get<0>(r3));
        t.cut_b.push_back(std::get<1>(r3));
        t.cut_e.push_back(std::get<2>(r3));
      }
    }
    t.cut_ptr.push_back((int)t.cut_a.size());
  }
  return t;
}

// Sec. III-B bisects buses; a three-phase bus has three nodes (Sec. III-A, after Eq. 3). The group
// graph has one edge per distinct pair of groups joined by a vertex branch, listed in ascending
// (min, max) order; its tree is expanded group by group (vertex B g + w at B pos(g) + w). Each
// tree node's cut columns factor the off-diagonal block of Eq. 3 exactly, H = G_lr = h_l h_r^T:
// one column per (left group A, right vertex y) of joined groups, h_r = e_y, h_l holding G[x, y]
// at A's B vertices, sorted by (position of A, position of y).
Tree build_block_tree(int n_vertex, int n_branch, const int32_t* from, const int32_t* to, int B, int levels,
                      int d_th) {
  EMT_REQUIRE(B >= 2 && n_vertex >= B && n_vertex % B == 0, EMT_ERR_INVALID,
              "block partition: the vertex count must be a positive multiple of nodes_per_bus");
  const int ng = n_vertex / B;
  std::vector<std::pair<int, int>> pairs;
  for (int e = 0; e < n_branch; ++e) {
    const int a = from[e], b = to[e];
    EMT_REQUIRE(a >= 0 && a < n_vertex && b >= -1 && b < n_vertex, EMT_ERR_INVALID, "branch endpoint out of range");
    if (b < 0 || a / B == b / B) continue;
    pairs.emplace_back(std::min(a / B, b / B), std::max(a / B, b / B));
  }
  std::sort(pairs.begin(), pairs.end());
  pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
  std::vector<int32_t> gf(pairs.size()), gt(pairs.size());
  for (size_t i = 0; i < pairs.size(); ++i) {
    gf[i] = pairs[i].first;
    gt[i] = pairs[i].second;
  }
  const Tree tg = build_tree(ng, (int)pairs.size(), gf.data(), gt.data(), levels, levels > 0 ? 0 : d_th / B);
  Tree t;
  t.n_bus = n_vertex;
  t.max_depth = tg.max_depth;
  t.parent = tg.parent;
  t.left = tg.left;
  t.right = tg.right;
  t.depth = tg.depth;
  t.leaves = tg.leaves;
  t.cut_w = B;
  t.perm.resize(n_vertex);
  t.pos.resize(n_vertex);
  for (int i = 0; i < ng; ++i)
    for (int w = 0; w < B; ++w) t.perm[B * i + w] = B * tg.perm[i] + w;
  for (int i = 0; i < n_vertex; ++i) t.pos[t.perm[i]] = i;
  const int nn = tg.n_node();
  t.lo.resize(nn);
  t.hi.resize(nn);
  for (int p = 0; p < nn; ++p) {
    t.lo[p] = B * tg.lo[p];
    t.hi[p] = B * tg.hi[p];
  }
  t.cut_ptr.push_back(0);
  for (int p = 0; p < nn; ++p) {
    if (tg.left[p] >= 0) {
      const int l = tg.left[p], r = tg.right[p];
      std::vector<std::pair<int, int>> cols;
      for (auto& pr : pairs) {
        const int pa = tg.pos[pr.first], pb = tg.pos[pr.second];
        int A, Bg;
        if (tg.lo[l] <= pa && pa < tg.hi[l] && tg.lo[r] <= pb && pb < tg.hi[r]) {
          A = pa;
          Bg = pb;
        } else if (tg.lo[l] <= pb && pb < tg.hi[l] && tg.lo[r] <= pa && pa < tg.hi[r]) {
          A = pb;
          Bg = pa;
        } else {
          continue;
        }
        for (int q = 0; q < B; ++q) cols.emplace_back(B * A, B * Bg + q);
      }
      std::sort(cols.begin(), cols.end());
      for (auto& c : cols) {
        t.cut_a.push_back(c.first);
        t.cut_b.push_back(c.second);
        t.cut_e.push_back(-1);
      }
    }
    t.cut_ptr.push_back((int)t.cut_a.size());
  }
  return t;
}

}  // namespace emt
