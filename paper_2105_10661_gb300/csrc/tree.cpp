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
#include <deque>
#include <map>
#include <tuple>

#include "internal.h"

namespace emt {
namespace {

struct Local {
  int n = 0;
  std::vector<std::vector<int>> nbr;   // ascending unique neighbours
  std::vector<std::vector<int>> wt;    // multiplicities
};

Local local_graph(const std::vector<int>& V, const std::vector<int>& gl2lo,
                  const std::vector<std::vector<int>>& adj_global) {
  Local g;
  g.n = (int)V.size();
  g.nbr.resize(g.n);
  g.wt.resize(g.n);
  for (int i = 0; i < g.n; ++i) {
    std::map<int, int> m;
    for (int u : adj_global[V[i]]) {
      int lu = gl2lo[u];
      if (lu < 0 || lu == i) continue;
      m[lu] += 1;
    }
    for (auto& kv : m) {
      g.nbr[i].push_back(kv.first);
      g.wt[i].push_back(kv.second);
    }
  }
  return g;
}

std::vector<int> bfs_dist(const Local& g, int s) {
  std::vector<int> d(g.n, -1);
  std::deque<int> q;
  d[s] = 0;
  q.push_back(s);
  while (!q.empty()) {
    int u = q.front();
    q.pop_front();
    for (int v : g.nbr[u])
      if (d[v] < 0) {
        d[v] = d[u] + 1;
        q.push_back(v);
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
  std::vector<int> order;
  order.reserve(g.n);
  auto run = [&](int r) {
    if (seen[r]) return;
    seen[r] = 1;
    std::deque<int> q;
    q.push_back(r);
    while (!q.empty()) {
      int u = q.front();
      q.pop_front();
      order.push_back(u);
      for (int v : g.nbr[u])
        if (!seen[v]) {
          seen[v] = 1;
          q.push_back(v);
        }
    }
  };
  run(start);
  for (int r = 0; r < g.n; ++r) run(r);
  return order;
}

void kernighan_lin(const Local& g, std::vector<int>& side, int passes) {
  const int n = g.n;
  const long long NEG = -(1LL << 60);
  std::vector<long long> D(n), vb(n);
  std::vector<char> locked(n);
  for (int pass = 0; pass < passes; ++pass) {
    for (int v = 0; v < n; ++v) {
      long long s = 0;
      for (size_t k = 0; k < g.nbr[v].size(); ++k)
        s += (side[g.nbr[v][k]] != side[v]) ? g.wt[v][k] : -g.wt[v][k];
      D[v] = s;
    }
    std::fill(locked.begin(), locked.end(), 0);
    int nA = 0;
    for (int v = 0; v < n; ++v) nA += side[v] == 0;
    int steps = std::min(nA, n - nA);
    std::vector<std::pair<int, int>> pairs;
    std::vector<long long> gains;
    for (int st = 0; st < steps; ++st) {
      int a = -1;
      long long best = NEG;
      for (int v = 0; v < n; ++v) {
        long long val = (side[v] == 0 && !locked[v]) ? D[v] : NEG;
        if (a < 0 || val > best) { best = val; a = v; }
      }
      for (int v = 0; v < n; ++v) vb[v] = (side[v] == 1 && !locked[v]) ? D[v] : NEG;
      long long wab = 0;
      for (size_t k = 0; k < g.nbr[a].size(); ++k) {
        int u = g.nbr[a][k];
        if (side[u] == 1 && !locked[u]) vb[u] -= 2LL * g.wt[a][k];
      }
      int b = -1;
      best = NEG;
      for (int v = 0; v < n; ++v)
        if (b < 0 || vb[v] > best) { best = vb[v]; b = v; }
      for (size_t k = 0; k < g.nbr[a].size(); ++k)
        if (g.nbr[a][k] == b) wab = g.wt[a][k];
      gains.push_back(D[a] + D[b] - 2 * wab);
      pairs.emplace_back(a, b);
      locked[a] = 1;
      locked[b] = 1;
      for (size_t k = 0; k < g.nbr[a].size(); ++k) {
        int x = g.nbr[a][k];
        if (!locked[x]) D[x] += (side[x] == 0) ? 2LL * g.wt[a][k] : -2LL * g.wt[a][k];
      }
      for (size_t k = 0; k < g.nbr[b].size(); ++k) {
        int y = g.nbr[b][k];
        if (!locked[y]) D[y] += (side[y] == 1) ? 2LL * g.wt[b][k] : -2LL * g.wt[b][k];
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
  std::vector<int> gl2lo(n_bus, -1);
  for (size_t i = 0; i < sets.size(); ++i) {
    const int n = (int)sets[i].size();
    bool split = n >= 2 && ((levels > 0 && depth[i] < levels) || (levels <= 0 && n > d_th));
    if (!split) continue;
    std::vector<int> V = sets[i];
    for (int k = 0; k < n; ++k) gl2lo[V[k]] = k;
    Local g = local_graph(V, gl2lo, adj);
    for (int k = 0; k < n; ++k) gl2lo[V[k]] = -1;
    int s = start_vertex(g);
    std::vector<int> order = growth_order(g, s);
    std::vector<int> side(n, 1);
    int nA = (n + 1) / 2;
    for (int k = 0; k < nA; ++k) side[order[k]] = 0;
    kernighan_lin(g, side, 4);
    std::vector<int> A, B;
    for (int k = 0; k < n; ++k) (side[k] == 0 ? A : B).push_back(V[k]);
    if (!(A.front() < B.front())) std::swap(A, B);
    int li = (int)sets.size();
    sets.push_back(A);
    sets.push_back(B);
    for (int c = 0; c < 2; ++c) {
      depth.push_back(depth[i] + 1);
      parent.push_back((int)i);
      left.push_back(-1);
      right.push_back(-1);
    }
    left[i] = li;
    right[i] = li + 1;
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

}  // namespace emt
