// Contraction-path search and slicing (Sec. 3.1).
//
// The paper finds a pseudo-optimal FLOP-minimising contraction sequence by
// recursive graph partitioning plus heuristics, and slices indices so that
// intermediates fit in memory.  Here:
//   * greedy_tree: pairwise greedy that contracts the connected pair with the
//     largest size reduction (|C| - |A| - |B| smallest), optional Gumbel noise
//     for randomised candidates; deterministic tie-break by tensor ids;
//   * bisect_tree: recursive min-cut bisection of the hypergraph (tensors =
//     vertices, indices = hyperedges) with Fiduccia-Mattheyses refinement,
//     finished by the greedy on small groups;
//   * choose_slices: repeatedly slices the index whose removal most lowers the
//     largest intermediate (then the total FLOPs) until the cap holds;
//   * reconfigure: local re-optimisation of a tree: every node's subtree is cut
//     into at most 8 frontier subtrees whose optimal contraction order (FLOPs,
//     with the intermediate-size cap as a constraint) is found by dynamic
//     programming over subsets and swapped in when cheaper.
// Labels may be hyperedges (batch labels sit on every projection leaf); a
// label stays open while a tensor outside the subtree still holds it or it is
// an output label.
#include <algorithm>
#include <array>
#include <cmath>
#include <limits>
#include <queue>
#include <functional>
#include <random>

#include "internal.h"

namespace tnq {

namespace {

using LC = std::vector<std::pair<int, int>>;  // (label, count in subtree), sorted by label

void merge_lc(const LC& a, const LC& b, LC* u) {
  u->clear();
  size_t i = 0, j = 0;
  while (i < a.size() || j < b.size()) {
    if (j == b.size() || (i < a.size() && a[i].first < b[j].first)) u->push_back(a[i++]);
    else if (i == a.size() || b[j].first < a[i].first) u->push_back(b[j++]);
    else {
      u->push_back({a[i].first, a[i].second + b[j].second});
      ++i;
      ++j;
    }
  }
}

void close_lc(const Hyper& h, const LC& u, LC* out) {
  out->clear();
  for (auto& e : u)
    if (h.is_output[e.first] || e.second < h.label_count[e.first]) out->push_back(e);
}

LC leaf_lc(const Hyper& h, int leaf, const std::vector<char>& sliced) {
  LC v;
  for (int l : h.leaf_labels[leaf])
    if (sliced.empty() || !sliced[l]) v.push_back({l, 1});
  return v;
}

struct Rng {
  std::mt19937_64 g;
  explicit Rng(uint64_t s) : g(s) {}
  double uni() { return (g() >> 11) * (1.0 / 9007199254740992.0); }
  uint64_t below(uint64_t n) { return g() % n; }
};

// Greedy over an initial set of (node id, labels) items, appending internal
// nodes to t; returns the root id.
int greedy_core(const Hyper& h, Tree* t, std::vector<std::pair<int, LC>> items, Rng* rng,
                double temperature) {
  if (items.empty()) return -1;
  struct Item {
    int id;
    LC lc;
    bool alive;
  };
  std::vector<Item> pool;
  for (auto& it : items) pool.push_back({it.first, it.second, true});
  std::vector<std::vector<int>> holders(h.n_labels);
  for (int i = 0; i < (int)pool.size(); ++i)
    for (auto& e : pool[i].lc) holders[e.first].push_back(i);
  struct Cand {
    double score;
    int i, j;
    bool operator<(const Cand& o) const {
      if (score != o.score) return score > o.score;  // min-heap
      if (i != o.i) return i > o.i;
      return j > o.j;
    }
  };
  std::priority_queue<Cand> heap;
  LC u, c;
  auto score = [&](int i, int j) {
    merge_lc(pool[i].lc, pool[j].lc, &u);
    close_lc(h, u, &c);
    double sa = std::ldexp(1.0, (int)pool[i].lc.size()), sb = std::ldexp(1.0, (int)pool[j].lc.size());
    double sc = std::ldexp(1.0, (int)c.size());
    double s = sc - sa - sb;
    if (temperature > 0) {
      double g = -std::log(-std::log(std::max(rng->uni(), 1e-300)));
      s -= temperature * g * std::max(sa, sb);
    }
    return s;
  };
  auto push_pairs_of = [&](int i) {
    std::vector<int> nb;
    for (auto& e : pool[i].lc)
      for (int j : holders[e.first])
        if (j != i && pool[j].alive) nb.push_back(j);
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    for (int j : nb) heap.push({score(std::min(i, j), std::max(i, j)), std::min(i, j), std::max(i, j)});
  };
  for (int i = 0; i < (int)pool.size(); ++i) push_pairs_of(i);
  int alive = (int)pool.size();
  while (alive > 1) {
    int a = -1, b = -1;
    while (!heap.empty()) {
      Cand cd = heap.top();
      heap.pop();
      if (pool[cd.i].alive && pool[cd.j].alive) {
        a = cd.i;
        b = cd.j;
        break;
      }
    }
    if (a < 0) {  // disconnected: outer product of the two smallest
      std::vector<int> live;
      for (int i = 0; i < (int)pool.size(); ++i)
        if (pool[i].alive) live.push_back(i);
      std::sort(live.begin(), live.end(), [&](int x, int y) {
        if (pool[x].lc.size() != pool[y].lc.size()) return pool[x].lc.size() < pool[y].lc.size();
        return x < y;
      });
      a = std::min(live[0], live[1]);
      b = std::max(live[0], live[1]);
    }
    merge_lc(pool[a].lc, pool[b].lc, &u);
    close_lc(h, u, &c);
    pool[a].alive = pool[b].alive = false;
    int id = t->n_leaves + (int)t->nodes.size();
    t->nodes.push_back({pool[a].id, pool[b].id});
    pool.push_back({id, c, true});
    int ni = (int)pool.size() - 1;
    for (auto& e : c) holders[e.first].push_back(ni);
    --alive;
    push_pairs_of(ni);
  }
  for (auto& p : pool)
    if (p.alive) return p.id;
  return -1;
}

// ---- FM bisection of a vertex subset
std::pair<std::vector<int>, std::vector<int>> fm_bisect(const Hyper& h, const std::vector<int>& S,
                                                        Rng* rng, double imbalance, int tries) {
  const int n = (int)S.size();
  // hyperedges restricted to S (labels with >= 2 pins in S)
  std::vector<int> lab_idx(h.n_labels, -1);
  std::vector<std::vector<int>> edges;
  std::vector<std::vector<int>> vedges(n);
  {
    std::vector<std::vector<int>> pins(h.n_labels);
    for (int v = 0; v < n; ++v)
      for (int l : h.leaf_labels[S[v]]) pins[l].push_back(v);
    for (int l = 0; l < h.n_labels; ++l)
      if (pins[l].size() >= 2) {
        int e = (int)edges.size();
        edges.push_back(pins[l]);
        for (int v : pins[l]) vedges[v].push_back(e);
      }
  }
  const int E = (int)edges.size();
  int lo = (int)std::floor(n * (0.5 - imbalance / 2)), hi = (int)std::ceil(n * (0.5 + imbalance / 2));
  lo = std::max(lo, 1);
  hi = std::min(hi, n - 1);
  std::vector<char> best_side;
  int best_cut = std::numeric_limits<int>::max();
  for (int t = 0; t < tries; ++t) {
    std::vector<char> side(n, 1);
    // BFS growth of side 0
    int target = n / 2, cnt = 0;
    std::vector<int> q;
    std::vector<char> seen(n, 0);
    while (cnt < target) {
      if (q.empty()) {
        std::vector<int> rest;
        for (int v = 0; v < n; ++v)
          if (!seen[v]) rest.push_back(v);
        int s = rest[rng->below(rest.size())];
        seen[s] = 1;
        q.push_back(s);
        side[s] = 0;
        ++cnt;
        continue;
      }
      int idx = (int)rng->below(std::min<size_t>(q.size(), 4));
      int v = q[idx];
      q.erase(q.begin() + idx);
      std::vector<int> nb;
      for (int e : vedges[v])
        for (int u : edges[e])
          if (!seen[u]) nb.push_back(u);
      std::shuffle(nb.begin(), nb.end(), rng->g);
      for (int u : nb) {
        if (cnt >= target) break;
        if (seen[u]) continue;
        seen[u] = 1;
        side[u] = 0;
        q.push_back(u);
        ++cnt;
      }
    }
    std::vector<std::array<int, 2>> pc(E);
    auto recount = [&]() {
      for (int e = 0; e < E; ++e) {
        pc[e] = {0, 0};
        for (int v : edges[e]) pc[e][side[v]]++;
      }
    };
    auto gain_of = [&](int v) {
      int g = 0, s = side[v];
      for (int e : vedges[v]) {
        if (pc[e][s] == 1 && pc[e][1 - s] > 0) ++g;
        if (pc[e][1 - s] == 0) --g;
      }
      return g;
    };
    recount();
    for (int pass = 0; pass < 12; ++pass) {
      std::vector<int> gain(n);
      for (int v = 0; v < n; ++v) gain[v] = gain_of(v);
      std::vector<char> locked(n, 0);
      std::vector<int> moves;
      int size0 = 0;
      for (int v = 0; v < n; ++v) size0 += side[v] == 0;
      int cur = 0, bestcum = 0, bestk = 0;
      for (int k = 0; k < n; ++k) {
        int bv = -1;
        double bkey = -1e300;
        for (int v = 0; v < n; ++v) {
          if (locked[v]) continue;
          int ns0 = size0 + (side[v] == 1 ? 1 : -1);
          if (ns0 < lo || ns0 > hi) continue;
          double key = gain[v] + 0.5 * rng->uni();
          if (key > bkey) {
            bkey = key;
            bv = v;
          }
        }
        if (bv < 0) break;
        int s = side[bv];
        cur += gain[bv];
        locked[bv] = 1;
        size0 += s == 1 ? 1 : -1;
        for (int e : vedges[bv]) {
          pc[e][s]--;
          pc[e][1 - s]++;
        }
        side[bv] = 1 - s;
        moves.push_back(bv);
        for (int e : vedges[bv])
          for (int u : edges[e])
            if (!locked[u]) gain[u] = gain_of(u);
        if (cur > bestcum) {
          bestcum = cur;
          bestk = k + 1;
        }
      }
      for (int k = (int)moves.size() - 1; k >= bestk; --k) {
        int v = moves[k], s = side[v];
        for (int e : vedges[v]) {
          pc[e][s]--;
          pc[e][1 - s]++;
        }
        side[v] = 1 - s;
      }
      if (bestcum <= 0) break;
    }
    int cut = 0;
    for (int e = 0; e < E; ++e) cut += pc[e][0] > 0 && pc[e][1] > 0;
    if (cut < best_cut) {
      best_cut = cut;
      best_side = side;
    }
  }
  std::vector<int> A, B;
  for (int v = 0; v < n; ++v) (best_side[v] == 0 ? A : B).push_back(S[v]);
  return {A, B};
}

int bisect_rec(const Hyper& h, Tree* t, const std::vector<int>& S, Rng* rng, double imbalance,
               int leaf_group) {
  if (S.size() == 1) return S[0];
  if ((int)S.size() <= leaf_group) {
    std::vector<std::pair<int, LC>> items;
    std::vector<char> none;
    for (int v : S) items.push_back({v, leaf_lc(h, v, none)});
    return greedy_core(h, t, items, rng, 0.0);
  }
  auto parts = fm_bisect(h, S, rng, imbalance, 2);
  if (parts.first.empty() || parts.second.empty()) {
    std::vector<std::pair<int, LC>> items;
    std::vector<char> none;
    for (int v : S) items.push_back({v, leaf_lc(h, v, none)});
    return greedy_core(h, t, items, rng, 0.0);
  }
  int a = bisect_rec(h, t, parts.first, rng, imbalance, leaf_group);
  int b = bisect_rec(h, t, parts.second, rng, imbalance, leaf_group);
  int id = t->n_leaves + (int)t->nodes.size();
  t->nodes.push_back({a, b});
  return id;
}

}  // namespace

Hyper make_hyper(const Network& net) {
  Hyper h;
  h.n_labels = net.n_labels;
  h.is_output = net.is_output;
  h.label_count.assign(net.n_labels, 0);
  for (auto& L : net.leaves) {
    std::vector<int> v = L.labels;
    std::sort(v.begin(), v.end());
    for (int l : v) h.label_count[l]++;
    h.leaf_labels.push_back(v);
  }
  return h;
}

// Node labels of every tree node (sliced labels removed); node ids as in Tree.
static void node_labels(const Hyper& h, const Tree& t, const std::vector<char>& sliced,
                        std::vector<LC>* labs, TreeCost* cost) {
  const int L = t.n_leaves, N = L + (int)t.nodes.size();
  labs->assign(N, LC());
  TreeCost c;
  for (int i = 0; i < L; ++i) {
    (*labs)[i] = leaf_lc(h, i, sliced);
    c.max_log2 = std::max(c.max_log2, (int)(*labs)[i].size());
  }
  LC u;
  for (int j = 0; j < (int)t.nodes.size(); ++j) {
    const LC& a = (*labs)[t.nodes[j].first];
    const LC& b = (*labs)[t.nodes[j].second];
    merge_lc(a, b, &u);
    close_lc(h, u, &(*labs)[L + j]);
    c.flops += 8.0 * std::ldexp(1.0, (int)u.size());
    c.bytes += 8.0 * (std::ldexp(1.0, (int)a.size()) + std::ldexp(1.0, (int)b.size()) +
                      std::ldexp(1.0, (int)(*labs)[L + j].size()));
    c.max_log2 = std::max(c.max_log2, (int)(*labs)[L + j].size());
  }
  if (cost) *cost = c;
}

TreeCost tree_cost(const Hyper& h, const Tree& t, const std::vector<char>& sliced) {
  std::vector<LC> labs;
  TreeCost c;
  node_labels(h, t, sliced, &labs, &c);
  return c;
}

Tree greedy_tree(const Hyper& h, const std::vector<char>& sliced, uint64_t seed, double temperature) {
  Tree t;
  t.n_leaves = (int)h.leaf_labels.size();
  Rng rng(seed);
  std::vector<std::pair<int, LC>> items;
  for (int i = 0; i < t.n_leaves; ++i) items.push_back({i, leaf_lc(h, i, sliced)});
  greedy_core(h, &t, items, &rng, temperature);
  return t;
}

Tree bisect_tree(const Hyper& h, uint64_t seed, double imbalance, int leaf_group) {
  Tree t;
  t.n_leaves = (int)h.leaf_labels.size();
  Rng rng(seed);
  std::vector<int> all(t.n_leaves);
  for (int i = 0; i < t.n_leaves; ++i) all[i] = i;
  bisect_rec(h, &t, all, &rng, imbalance, leaf_group);
  return t;
}

std::vector<int> choose_slices(const Hyper& h, const Tree& t, int cap_log2, bool* feasible) {
  std::vector<char> sliced(h.n_labels, 0);
  std::vector<int> chosen;
  *feasible = true;
  for (int iter = 0; iter < 64; ++iter) {
    std::vector<LC> labs;
    TreeCost c;
    node_labels(h, t, sliced, &labs, &c);
    if (c.max_log2 <= cap_log2) return chosen;
    std::vector<char> cand(h.n_labels, 0);
    for (auto& lc : labs)
      if ((int)lc.size() > cap_log2)
        for (auto& e : lc)
          if (!h.is_output[e.first]) cand[e.first] = 1;
    int best = -1;
    double best_flops = 0;
    int best_max = 1 << 30;
    for (int l = 0; l < h.n_labels; ++l) {
      if (!cand[l]) continue;
      sliced[l] = 1;
      TreeCost c2 = tree_cost(h, t, sliced);
      sliced[l] = 0;
      if (c2.max_log2 < best_max || (c2.max_log2 == best_max && c2.flops < best_flops)) {
        best = l;
        best_max = c2.max_log2;
        best_flops = c2.flops;
      }
    }
    if (best < 0) break;
    sliced[best] = 1;
    chosen.push_back(best);
  }
  if (tree_cost(h, t, sliced).max_log2 > cap_log2) *feasible = false;
  return chosen;
}

namespace {

struct Bits256 {
  uint64_t w[4] = {0, 0, 0, 0};
  void set(int i) { w[i >> 6] |= uint64_t(1) << (i & 63); }
  Bits256 operator|(const Bits256& o) const {
    Bits256 r;
    for (int i = 0; i < 4; ++i) r.w[i] = w[i] | o.w[i];
    return r;
  }
  Bits256 operator&(const Bits256& o) const {
    Bits256 r;
    for (int i = 0; i < 4; ++i) r.w[i] = w[i] & o.w[i];
    return r;
  }
  int count() const { return __builtin_popcountll(w[0]) + __builtin_popcountll(w[1]) + __builtin_popcountll(w[2]) +
                             __builtin_popcountll(w[3]); }
};

}  // namespace

int reconfigure(const Hyper& h, Tree* t, const std::vector<char>& sliced, int cap_log2, int max_frontier,
                int sweeps) {
  const int L = t->n_leaves;
  const int N = L + (int)t->nodes.size();
  if (t->nodes.empty()) return 0;
  int improved = 0;
  for (int sw = 0; sw < sweeps; ++sw) {
    std::vector<LC> labs;
    node_labels(h, *t, sliced, &labs, nullptr);
    std::vector<int> left(N, -1), right(N, -1);
    for (int j = 0; j < (int)t->nodes.size(); ++j) {
      left[L + j] = t->nodes[j].first;
      right[L + j] = t->nodes[j].second;
    }
    const int root = N - 1;
    int changed = 0;
    // visit internal nodes top-down so re-optimised regions are used as given
    for (int v = N - 1; v >= L; --v) {
      // frontier: expand the largest internal member until max_frontier members
      std::vector<int> front = {left[v], right[v]};
      std::vector<int> inner = {v};
      while ((int)front.size() < max_frontier) {
        int bi = -1;
        size_t bs = 0;
        for (int i = 0; i < (int)front.size(); ++i)
          if (front[i] >= L && (bi < 0 || labs[front[i]].size() > bs)) {
            bi = i;
            bs = labs[front[i]].size();
          }
        if (bi < 0) break;
        const int u = front[bi];
        inner.push_back(u);
        front[bi] = left[u];
        front.push_back(right[u]);
      }
      const int k = (int)front.size();
      if (k < 3) continue;
      // local label bitsets
      std::vector<int> ids;
      for (int f : front)
        for (auto& e : labs[f]) ids.push_back(e.first);
      std::sort(ids.begin(), ids.end());
      ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
      if (ids.size() > 256) continue;
      auto bit_of = [&](int l) { return int(std::lower_bound(ids.begin(), ids.end(), l) - ids.begin()); };
      std::vector<Bits256> in1(k);
      for (int i = 0; i < k; ++i)
        for (auto& e : labs[front[i]]) in1[i].set(bit_of(e.first));
      Bits256 vout;
      for (auto& e : labs[v]) {
        auto it = std::lower_bound(ids.begin(), ids.end(), e.first);
        if (it != ids.end() && *it == e.first) vout.set(int(it - ids.begin()));
      }
      const int full = (1 << k) - 1;
      std::vector<Bits256> in(1 << k), open(1 << k);
      for (int S = 1; S <= full; ++S) {
        const int low = __builtin_ctz(S);
        in[S] = in[S & (S - 1)] | in1[low];
      }
      for (int S = 1; S <= full; ++S) open[S] = in[S] & (in[full & ~S] | vout);
      std::vector<double> cost(1 << k, 1e300);
      std::vector<int> split(1 << k, 0);
      for (int i = 0; i < k; ++i) cost[1 << i] = 0;
      for (int S = 1; S <= full; ++S) {
        if (__builtin_popcount(S) < 2) continue;
        if (S != full && open[S].count() > cap_log2) continue;
        const int low = S & -S;
        for (int A = (S - 1) & S; A > 0; A = (A - 1) & S) {
          if (!(A & low)) continue;
          const int B = S ^ A;
          if (cost[A] >= 1e299 || cost[B] >= 1e299) continue;
          const double c = cost[A] + cost[B] + 8.0 * std::ldexp(1.0, (open[A] | open[B]).count());
          if (c < cost[S]) {
            cost[S] = c;
            split[S] = A;
          }
        }
      }
      // current cost of the region between v and its frontier
      double cur = 0;
      for (int u : inner) {
        LC uu;
        merge_lc(labs[left[u]], labs[right[u]], &uu);
        cur += 8.0 * std::ldexp(1.0, (int)uu.size());
      }
      if (!(cost[full] < cur * (1.0 - 1e-9))) continue;
      // rebuild the region with the inner node ids (v stays the region's root)
      std::vector<int> pool(inner.begin() + 1, inner.end());
      std::function<int(int, int)> build = [&](int S, int as) -> int {
        if (__builtin_popcount(S) == 1) return front[__builtin_ctz(S)];
        const int A = split[S], B = S ^ A;
        const int node = as >= 0 ? as : pool.back();
        if (as < 0) pool.pop_back();
        const int a = build(A, -1), b = build(B, -1);
        left[node] = a;
        right[node] = b;
        return node;
      };
      build(full, v);
      ++changed;
      // label sets of rebuilt inner nodes: recompute the region bottom-up
      std::function<void(int)> relabel = [&](int u) {
        if (u < L) return;
        relabel(left[u]);
        relabel(right[u]);
        LC uu;
        merge_lc(labs[left[u]], labs[right[u]], &uu);
        close_lc(h, uu, &labs[u]);
      };
      relabel(v);
    }
    if (!changed) break;
    improved += changed;
    // re-linearise in post order from the root
    Tree nt;
    nt.n_leaves = L;
    std::vector<int> newid(N, -1);
    for (int i = 0; i < L; ++i) newid[i] = i;
    std::vector<std::pair<int, int>> stack;  // (node, state)
    stack.push_back({root, 0});
    while (!stack.empty()) {
      auto& top = stack.back();
      const int u = top.first;
      if (u < L) {
        stack.pop_back();
        continue;
      }
      if (top.second == 0) {
        top.second = 1;
        stack.push_back({left[u], 0});
      } else if (top.second == 1) {
        top.second = 2;
        stack.push_back({right[u], 0});
      } else {
        newid[u] = L + (int)nt.nodes.size();
        nt.nodes.push_back({newid[left[u]], newid[right[u]]});
        stack.pop_back();
      }
    }
    *t = nt;
  }
  return improved;
}

}  // namespace tnq
