// Plan = network + contraction tree + sliced labels + per-step GEMM layouts +
// workspace layout.  Host only.
//
// Each internal tree node is one pairwise contraction (Sec. 3.1).  Its labels
// split into H (batch: held by both operands and kept), K (contracted), M
// (operand A only), N (operand B only).  The step runs as a batched complex
// GEMM C[h][m][n] = sum_k A[h][m][k] B[h][n][k]; operands whose stored label
// order differs from [K][M|N][H] (bit 0 first) are bit-permuted first, and the
// output is stored as [N][M][H] so that the next step often needs no permute.
// Sliced labels are fixed per pass (Sec. 3.1 slicing); only leaves hold them,
// and a leaf holding one is always gathered through the permute kernel.
#include <algorithm>
#include <atomic>
#include <thread>
#include <chrono>
#include <cmath>
#include <map>
#include <random>

#include <set>

#include "internal.h"
#include "splitk.h"
#include "gemm_tc.cuh"
#include "mlp.h"

namespace tnq {

namespace {

// Largest slice-batched output (log2 elements, sliced indices included).
constexpr int kSliceBatchMaxLog2 = 16;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool contains(const std::vector<int>& v, int l) { return std::find(v.begin(), v.end(), l) != v.end(); }

}  // namespace

void layout_steps(Plan* p) {
  const Hyper& h = p->hyper;
  const Tree& t = p->tree;
  const int L = t.n_leaves;
  p->tensors.assign(L + t.nodes.size(), TensorSlot());
  for (int i = 0; i < L; ++i) {
    auto& ts = p->tensors[i];
    ts.leaf = true;
    ts.labels = p->net.leaves[i].labels;  // storage order, may include sliced labels
    ts.rank = (int)ts.labels.size();
  }
  // ---- classes of the steps: folded (constant subtree), slice-batched (small
  // slice-dependent subtree run once with its sliced indices kept), or
  // neither.  A tensor's "sliced count" is the number of distinct sliced
  // indices in its subtree; an unsliced subtree result has the rank of its
  // open indices.
  const int NT = L + (int)t.nodes.size();
  std::vector<std::set<int>> sub_sliced(NT);
  std::vector<char> is_const(NT, 0), is_batched(NT, 0);
  std::vector<int> open_rank(NT, 0);
  {
    std::vector<std::map<int, int>> c2(NT);
    for (int i = 0; i < L; ++i) {
      const Leaf& lf = p->net.leaves[i];
      is_const[i] = lf.kind == LEAF_STATIC;
      for (int l : lf.labels) {
        if (p->sliced[l]) {
          sub_sliced[i].insert(l);
          is_const[i] = 0;
        } else {
          c2[i][l] = 1;
        }
      }
      open_rank[i] = (int)c2[i].size();
    }
    for (int j = 0; j < (int)t.nodes.size(); ++j) {
      const int x = t.nodes[j].first, y = t.nodes[j].second, id = L + j;
      for (auto& e : c2[x]) c2[id][e.first] += e.second;
      for (auto& e : c2[y]) c2[id][e.first] += e.second;
      int r = 0;
      for (auto& e : c2[id])
        if (h.is_output[e.first] || e.second < h.label_count[e.first]) ++r;
      open_rank[id] = r;
      c2[x].clear();
      c2[y].clear();
      sub_sliced[id] = sub_sliced[x];
      sub_sliced[id].insert(sub_sliced[y].begin(), sub_sliced[y].end());
      is_const[id] = is_const[x] && is_const[y];
      // children must be leaves, slice-free steps or slice-batched steps
      auto ready = [&](int c) { return c < L || sub_sliced[c].empty() || is_batched[c]; };
      is_batched[id] = !sub_sliced[id].empty() && id != L + (int)t.nodes.size() - 1 && ready(x) && ready(y) &&
                       open_rank[id] + (int)sub_sliced[id].size() <= std::min(kSliceBatchMaxLog2, p->cap_log2);
    }
  }
  // subtree label counts for open/closed decisions
  std::vector<std::map<int, int>> cnt(L + t.nodes.size());
  for (int i = 0; i < L; ++i)
    for (int l : p->net.leaves[i].labels)
      if (!p->sliced[l]) cnt[i][l] = 1;
  auto eff = [&](int id) {
    std::vector<int> v;
    for (int l : p->tensors[id].labels)
      if (!p->sliced[l]) v.push_back(l);
    return v;
  };
  p->steps.clear();
  int max_op = 0;
  for (int j = 0; j < (int)t.nodes.size(); ++j) {
    int x = t.nodes[j].first, y = t.nodes[j].second, id = L + j;
    for (auto& e : cnt[x]) cnt[id][e.first] += e.second;
    for (auto& e : cnt[y]) cnt[id][e.first] += e.second;
    std::vector<int> out_set;
    for (auto& e : cnt[id])
      if (h.is_output[e.first] || e.second < h.label_count[e.first]) out_set.push_back(e.first);
    // a slice-batched step keeps every sliced index of its operands (as a
    // batch index when both hold it)
    std::vector<int> lx = is_batched[id] ? p->tensors[x].labels : eff(x);
    std::vector<int> ly = is_batched[id] ? p->tensors[y].labels : eff(y);
    if (is_batched[id])
      for (int l : sub_sliced[id]) out_set.push_back(l);
    // A = operand with fewer elements (it is the one expanded for the tensor cores)
    bool x_is_a = lx.size() <= ly.size();
    int a = x_is_a ? x : y, b = x_is_a ? y : x;
    std::vector<int> la = x_is_a ? lx : ly, lb = x_is_a ? ly : lx;
    // K and H orders follow the larger operand, except in dot-shaped steps
    // (at most 8 x 8 outputs per batch entry, at least 2^10 K values): there they
    // follow the operand whose stored layout starts with the longer run of K
    // labels, which the dot kernel then reads in place
    int nk_all = 0, nm = 0, nn = 0;
    for (int l : lb)
      if (contains(la, l) && !contains(out_set, l)) ++nk_all;
    for (int l : la)
      if (!contains(lb, l)) ++nm;
    for (int l : lb)
      if (!contains(la, l)) ++nn;
    auto low_k_run = [&](int id) {
      int run = 0;
      for (int l : p->tensors[id].labels) {
        if (p->sliced[l] || !contains(la, l) || !contains(lb, l) || contains(out_set, l)) break;
        ++run;
      }
      return run;
    };
    const bool dot_shaped = nm <= 3 && nn <= 3 && nk_all >= 10;
    const bool anchor_a = dot_shaped && low_k_run(a) > low_k_run(b);
    const std::vector<int>& anchor = anchor_a ? la : lb;
    const std::vector<int>& other = anchor_a ? lb : la;
    std::vector<int> K, Hh, M, N;
    for (int l : anchor)
      if (contains(other, l)) (contains(out_set, l) ? Hh : K).push_back(l);
    for (int l : la)
      if (!contains(lb, l)) M.push_back(l);
    for (int l : lb)
      if (!contains(la, l)) N.push_back(l);
    Step s;
    s.a = a;
    s.b = b;
    s.out = id;
    s.nH = (int)Hh.size();
    s.nM = (int)M.size();
    s.nN = (int)N.size();
    s.nK = (int)K.size();
    s.a_req = K;
    s.a_req.insert(s.a_req.end(), M.begin(), M.end());
    s.a_req.insert(s.a_req.end(), Hh.begin(), Hh.end());
    s.b_req = K;
    s.b_req.insert(s.b_req.end(), N.begin(), N.end());
    s.b_req.insert(s.b_req.end(), Hh.begin(), Hh.end());
    s.out_labels = N;
    s.out_labels.insert(s.out_labels.end(), M.begin(), M.end());
    s.out_labels.insert(s.out_labels.end(), Hh.begin(), Hh.end());
    s.perm_a = p->tensors[a].labels != s.a_req;
    s.perm_b = p->tensors[b].labels != s.b_req;
    s.flops = 8.0 * std::ldexp(1.0, s.nH + s.nM + s.nN + s.nK);
    s.fold = is_const[id];
    s.sliced_batch = is_batched[id];
    auto& ts = p->tensors[id];
    ts.labels = s.out_labels;
    ts.rank = (int)s.out_labels.size();
    max_op = std::max({max_op, (int)s.a_req.size(), (int)s.b_req.size()});
    p->steps.push_back(s);
    cnt[x].clear();
    cnt[y].clear();
  }
  p->root = L + (int)t.nodes.size() - 1;
  p->max_operand_log2 = max_op;
  // slice dependence: a leaf depends on the slice when it holds a sliced label,
  // a step output when either operand does
  std::vector<char> dep(p->tensors.size(), 0);
  for (int i = 0; i < L; ++i)
    for (int l : p->net.leaves[i].labels)
      if (p->sliced[l]) dep[i] = 1;
  for (auto& s : p->steps) {
    dep[s.out] = dep[s.a] || dep[s.b];
    s.invariant = !dep[s.out];
  }
  // lifetime class of a step: 0 folded (at bind), 1 once per batch, 2 per
  // slice; an output read by a step of a later class persists outside the
  // reusable arena (folded outputs for the binding, the others for the batch)
  auto cls = [&](const Step& s) { return s.fold ? 0 : s.once() ? 1 : 2; };
  std::vector<int> out_cls(p->tensors.size(), -1);
  for (auto& s : p->steps) out_cls[s.out] = cls(s);
  std::vector<char> pinned(p->tensors.size(), 0);
  for (auto& s : p->steps) {
    if (s.a >= L && out_cls[s.a] < cls(s)) pinned[s.a] = 1;
    if (s.b >= L && out_cls[s.b] < cls(s)) pinned[s.b] = 1;
  }

  // ---- workspace: [leaves][arena of intermediates][scratch A][scratch B][acc][misc]
  size_t off = 0;
  for (int i = 0; i < L; ++i) {
    off = align_up(off, 256);
    p->tensors[i].offset = off;
    off += (size_t(8) << p->tensors[i].rank);
  }
  p->ws_leaves = 0;
  off = align_up(off, 256);
  p->ws_persist = off;
  for (size_t id = L; id < p->tensors.size(); ++id)
    if (pinned[id]) {
      off = align_up(off, 256);
      p->tensors[id].offset = off;
      off += size_t(8) << p->tensors[id].rank;
    }
  p->ws_persist_bytes = off - p->ws_persist;
  size_t arena_base = align_up(off, 256);
  // first-fit arena over step outputs with liveness (an output lives until the
  // step that consumes it; the root lives to the end)
  struct Blk {
    size_t off, size;
    int owner;
  };
  std::vector<Blk> live;
  size_t arena_top = 0;
  auto alloc = [&](size_t sz, int owner) {
    sz = align_up(sz, 256);
    std::sort(live.begin(), live.end(), [](const Blk& u, const Blk& v) { return u.off < v.off; });
    size_t cur = 0;
    for (auto& bk : live) {
      if (bk.off >= cur + sz) break;
      cur = std::max(cur, bk.off + bk.size);
    }
    live.push_back({cur, sz, owner});
    arena_top = std::max(arena_top, cur + sz);
    return cur;
  };
  auto release = [&](int owner) {
    live.erase(std::remove_if(live.begin(), live.end(), [&](const Blk& bk) { return bk.owner == owner; }),
               live.end());
  };
  for (auto& s : p->steps) {
    if (!pinned[s.out]) p->tensors[s.out].offset = arena_base + alloc(size_t(8) << p->tensors[s.out].rank, s.out);
    if (s.a >= L) release(s.a);
    if (s.b >= L) release(s.b);
  }
  p->ws_arena = arena_base;
  p->ws_arena_bytes = arena_top;
  off = align_up(arena_base + arena_top, 1024);
  // scratch: A expanded to 2Mx2K reals with a hi/lo split (32 B per complex
  // element, worst case), B with a hi/lo split (16 B per complex element)
  size_t max_a = 0, max_b = 0;
  for (auto& s : p->steps) {
    max_a = std::max(max_a, size_t(1) << s.a_req.size());
    max_b = std::max(max_b, size_t(1) << s.b_req.size());
  }
  p->ws_scratch_a = off;
  off = align_up(off + 32 * max_a + 4096, 1024);
  p->ws_scratch_b = off;
  off = align_up(off + 16 * max_b + 4096, 1024);
  p->ws_scratch_bytes = 32 * max_a + 16 * max_b;
  // FP32 partial products of split-K steps (largest need over steps and kernels)
  size_t max_part = 0;
  for (auto& s : p->steps) {
    int sp = std::max({simt_splits(s.nH, s.nM, s.nN, s.nK), tc_splits(s.nH, s.nM, s.nN, s.nK, true),
                       tc_splits(s.nH, s.nM, s.nN, s.nK, false), rows_splits(s.nH, s.nM, s.nN, s.nK)});
    if (use_dot(s.nM, s.nN, s.nK)) sp = std::max(sp, dot_splits(s.nH, s.nM, s.nN, s.nK));
    if (sp > 1 || use_dot(s.nM, s.nN, s.nK))
      max_part = std::max(max_part, size_t(sp) * 8 * (size_t(1) << (s.nH + s.nM + s.nN)));
  }
  p->ws_partial = off;
  off = align_up(off + max_part + 256, 1024);
  p->ws_acc = off;
  off = align_up(off + 16 * (size_t(1) << p->tensors[p->root].rank), 256);
  // trajectory program tables
  for (size_t i = 0; i < p->traj_leaves.size(); ++i) p->traj_leaves[i].out_offset = (long long)p->tensors[p->traj_leaf_ids[i]].offset;
  p->ws_traj = off;
  off = align_up(off + sizeof(TrajLeafDesc) * p->traj_leaves.size(), 256);
  p->ws_traj_factors = off;
  off = align_up(off + sizeof(TrajFactor) * p->traj_factors.size(), 256);
  p->ws_traj_mats = off;
  off = align_up(off + 16 * p->traj_mats.size(), 256);
  p->ws_traj_cumq = off;
  off = align_up(off + 8 * p->traj_cumq.size(), 256);
  p->ws_dedup_picks = off;
  off = align_up(off + (p->chan_cumq.size() << p->traj_log2), 256);
  p->ws_dedup_w = off;
  off = align_up(off + (p->chan_cumq.empty() ? 0 : size_t(8) << p->traj_log2), 256);
  p->ws_misc = off;
  const size_t per = size_t(1) << p->batch_log2;
  const size_t n_open = p->net.open_qubits.size();
  p->ws_bits = off + 256;
  p->ws_out_stage = align_up(p->ws_bits + size_t(p->net.row_len) * per, 256);
  p->ws_psum = align_up(p->ws_out_stage + std::max((16 * per) << n_open, size_t(16) << p->traj_log2), 256);
  p->ws_p2sum = align_up(p->ws_psum + 8 * per, 256);
  p->ws_qtab = align_up(p->ws_p2sum + 8 * per, 256);
  p->ws_picks = align_up(p->ws_qtab + 4 * (p->net.proj_src.size() + n_open), 256);
  off = align_up(p->ws_picks + p->picks.size(), 256);
  p->ws_total = off;
}

// Device program of the trajectory leaves: per leaf its factors in circuit
// order; gate matrices as given, channels as their Kraus operators rescaled by
// 1/sqrt(q_k) with the cumulative q table (summed in index order).
static void build_traj_program(const Circuit& c, Plan* p) {
  p->traj_leaves.clear();
  p->traj_leaf_ids.clear();
  p->traj_factors.clear();
  p->traj_mats.clear();
  p->traj_cumq.clear();
  p->chan_cumq.assign(c.n_channels, {});
  for (const COp& op : c.ops)
    if (op.channel && !op.selector && op.channel_index >= 0) {
      double acc = 0;
      for (double q : op.kraus_q) p->chan_cumq[op.channel_index].push_back(acc += q);
    }
  auto push_mat = [&](const std::vector<cd>& m) {
    int idx = (int)(p->traj_mats.size() / 16);
    std::vector<cd> e(16, cd(0, 0));
    for (size_t i = 0; i < m.size() && i < 16; ++i) e[i] = m[i];
    p->traj_mats.insert(p->traj_mats.end(), e.begin(), e.end());
    return idx;
  };
  for (int li = 0; li < (int)p->net.leaves.size(); ++li) {
    const Leaf& L = p->net.leaves[li];
    if (L.kind != LEAF_TRAJ) continue;
    TrajLeafDesc d;
    d.n_slots = L.n_slots;
    d.in_fixed_mask = L.in_fixed_mask;
    d.n_factors = (int)L.factors.size();
    d.factor_off = (int)p->traj_factors.size();
    d.out_offset = 0;
    d.nfree = 0;
    for (int s = 0; s < L.n_slots; ++s) d.nfree += !((L.in_fixed_mask >> s) & 1);
    for (const GroupFactor& g : L.factors) {
      const COp& op = c.ops[g.op];
      TrajFactor f;
      f.channel = op.channel ? 1 : 0;
      f.arity = (int)op.qubits.size();
      f.slot_mask = g.slot_mask;
      f.swap = g.swap ? 1 : 0;
      f.n_ops = 0;
      f.cum_off = 0;
      f.chan_index = op.channel_index;
      if (!op.channel) {
        f.mat_off = push_mat(op.mats[0]);
      } else if (op.selector) {
        f.channel = 2;
        f.n_ops = (int)op.mats.size();
        f.chan_index = op.selector_index;
        for (int k = 0; k < f.n_ops; ++k) {
          int idx = push_mat(op.mats[k]);
          if (k == 0) f.mat_off = idx;
        }
      } else {
        f.n_ops = (int)op.mats.size();
        f.cum_off = (int)p->traj_cumq.size();
        double acc = 0;
        for (int k = 0; k < f.n_ops; ++k) {
          acc += op.kraus_q[k];
          p->traj_cumq.push_back(acc);
          std::vector<cd> a = op.mats[k];
          const double s = op.kraus_q[k] > 0 ? 1.0 / std::sqrt(op.kraus_q[k]) : 0.0;
          for (auto& z : a) z *= s;
          int idx = push_mat(a);
          if (k == 0) f.mat_off = idx;
        }
      }
      p->traj_factors.push_back(f);
    }
    p->traj_leaves.push_back(d);
    p->traj_leaf_ids.push_back(li);
  }
}

// Per-step features for the cost model (16 floats per step): log2 sizes of the
// batch, row, column and contracted dimensions and of the work, operand and
// output elements (scaled by 1/32), whether each operand is permuted, which
// kernel the executor dispatches the step to at this precision, log2 of the
// algorithmic bytes, and whether it is the root step.
void step_features(const Plan& p, int precision, std::vector<float>* out) {
  out->clear();
  for (size_t i = 0; i < p.steps.size(); ++i) {
    const Step& s = p.steps[i];
    const int work = s.nH + s.nM + s.nN + s.nK;
    const bool tc = precision != TNQ_PREC_FP32 && !skinny(s.nM, s.nN, s.nK) &&
                    tc_gemm_supported(1 << s.nM, 1 << s.nN, 1 << s.nK, precision) && work >= 18;
    const bool dot = !tc && use_dot(s.nM, s.nN, s.nK);
    const bool rows = !tc && !dot && skinny(s.nM, s.nN, s.nK);
    const bool simt = !tc && !dot && !rows;
    const double bytes = 8.0 * (std::ldexp(1.0, (int)s.a_req.size()) + std::ldexp(1.0, (int)s.b_req.size()) +
                                std::ldexp(1.0, (int)s.out_labels.size()));
    const float f[kStepFeatures] = {s.nH / 32.f,
                                    s.nM / 32.f,
                                    s.nN / 32.f,
                                    s.nK / 32.f,
                                    work / 32.f,
                                    float(s.a_req.size()) / 32.f,
                                    float(s.b_req.size()) / 32.f,
                                    float(s.out_labels.size()) / 32.f,
                                    s.perm_a ? 1.f : 0.f,
                                    s.perm_b ? 1.f : 0.f,
                                    tc ? 1.f : 0.f,
                                    rows ? 1.f : 0.f,
                                    dot ? 1.f : 0.f,
                                    simt ? 1.f : 0.f,
                                    float(std::log2(bytes)) / 32.f,
                                    i + 1 == p.steps.size() ? 1.f : 0.f};
    out->insert(out->end(), f, f + kStepFeatures);
  }
}

tnq_status make_plan(const Circuit& c, const tnq_plan_opts& o, Plan* p, const NetworkSpec& spec) {
  return make_plan_ranked(c, o, p, nullptr, spec);
}

tnq_status make_plan_ranked(const Circuit& c, const tnq_plan_opts& o, Plan* p, const CandidateRanker* ranker,
                            const NetworkSpec& spec) {
  auto t0 = std::chrono::steady_clock::now();
  if (o.batch_log2 < 0 || o.batch_log2 > 16 || o.traj_log2 < 0 || o.traj_log2 > 16)
    return fail(TNQ_ERR_INVALID_ARG, "batch_log2/traj_log2 must be in [0, 16]");
  if (o.max_intermediate_log2 < 1 || o.max_intermediate_log2 > 31)
    return fail(TNQ_ERR_INVALID_ARG, "max_intermediate_log2 must be in [1, 31]");
  p->batch_log2 = o.batch_log2;
  p->cap_log2 = o.max_intermediate_log2;
  p->traj_log2 = (c.n_channels > 0 || c.n_selectors > 0) ? o.traj_log2 : 0;
  tnq_status st = build_network(c, p->batch_log2, p->traj_log2, spec.open, spec.row_len, &p->net);
  if (st != TNQ_OK) return st;
  p->hyper = make_hyper(p->net);
  build_traj_program(c, p);
  const Hyper& h = p->hyper;
  std::vector<Tree> cands;
  int mode = o.path_mode;
  int nc = std::max(1, o.n_candidates);
  if (mode == TNQ_PATH_GREEDY || mode == TNQ_PATH_BEST || mode == TNQ_PATH_LEARNED)
    cands.push_back(greedy_tree(h, {}, o.seed, 0.0));
  if (mode == TNQ_PATH_BISECT || mode == TNQ_PATH_BEST || mode == TNQ_PATH_LEARNED) {
    std::mt19937_64 g(o.seed ^ 0x5bd1e995ULL);
    struct Spec {
      uint64_t seed;
      double imb;
      int grp;
    };
    std::vector<Spec> specs(nc);
    for (int i = 0; i < nc; ++i) {
      specs[i].imb = 0.05 + 0.6 * ((g() >> 11) * (1.0 / 9007199254740992.0));
      specs[i].grp = 4 + int(g() % 12);
      specs[i].seed = g();
    }
    size_t base = cands.size();
    cands.resize(base + nc);
    int nthreads = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 32u);
    std::atomic<int> next(0);
    std::vector<std::thread> pool;
    for (int t = 0; t < std::min(nthreads, nc); ++t)
      pool.emplace_back([&] {
        for (int i = next++; i < nc; i = next++) cands[base + i] = bisect_tree(h, specs[i].seed, specs[i].imb, specs[i].grp);
      });
    for (auto& th : pool) th.join();
    for (int i = 0; i < nc / 4; ++i) cands.push_back(greedy_tree(h, {}, g(), 0.3 + 0.2 * (i % 4)));
  }
  if (cands.empty()) return fail(TNQ_ERR_INVALID_ARG, "unknown path_mode");
  // Evaluate candidates (slicing included) on host threads; each candidate's
  // result depends only on its own seed, and ties go to the lowest index, so
  // the choice is deterministic.
  const int NC = (int)cands.size();
  std::vector<double> totals(NC, -1.0);
  std::vector<std::vector<int>> slices(NC);
  // Per candidate: re-optimise the unsliced tree locally, choose the slices,
  // then re-optimise again under the size cap with the sliced labels fixed.
  auto eval = [&](int i) {
    bool feas = false;
    reconfigure(h, &cands[i], std::vector<char>(h.n_labels, 0), 64, 8, 4);
    std::vector<int> sl = choose_slices(h, cands[i], o.max_intermediate_log2, &feas);
    if (!feas) return;
    std::vector<char> sv(h.n_labels, 0);
    for (int l : sl) sv[l] = 1;
    // local re-optimisation of the sliced tree under the same size cap
    reconfigure(h, &cands[i], sv, o.max_intermediate_log2, 8, 6);
    TreeCost tc = tree_cost(h, cands[i], sv);
    if (tc.max_log2 > o.max_intermediate_log2) return;
    totals[i] = tc.flops * std::ldexp(1.0, (int)sl.size());
    slices[i] = sl;
  };
  int nthreads = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 32u);
  nthreads = std::min(nthreads, NC);
  if (nthreads <= 1) {
    for (int i = 0; i < NC; ++i) eval(i);
  } else {
    std::atomic<int> next(0);
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t)
      pool.emplace_back([&] {
        for (int i = next++; i < NC; i = next++) eval(i);
      });
    for (auto& th : pool) th.join();
  }
  double best_total = 0;
  int best = -1;
  std::vector<int> best_slices;
  for (int i = 0; i < NC; ++i) {
    if (totals[i] < 0) continue;
    if (best < 0 || totals[i] < best_total) {
      best = i;
      best_total = totals[i];
      best_slices = slices[i];
    }
  }
  // record every candidate's sliced flops; a ranker may override the choice
  p->cand_flops = totals;
  p->cand_pred.assign(NC, -1.0);
  p->cand_flopmin = best;
  if (best >= 0 && ranker) {
    int pick = -1;
    double pick_t = 0;
    for (int i = 0; i < NC; ++i) {
      if (totals[i] < 0) continue;
      Plan tmp;
      tmp.net = p->net;
      tmp.hyper = p->hyper;
      tmp.tree = cands[i];
      tmp.batch_log2 = p->batch_log2;
      tmp.cap_log2 = p->cap_log2;
      tmp.traj_log2 = p->traj_log2;
      tmp.sliced.assign(h.n_labels, 0);
      tmp.slice_labels = slices[i];
      for (int l : slices[i]) tmp.sliced[l] = 1;
      layout_steps(&tmp);
      double t = 0;
      tnq_status rs = (*ranker)(tmp, &t);
      if (rs != TNQ_OK) return rs;
      t *= std::ldexp(1.0, (int)slices[i].size());
      p->cand_pred[i] = t;
      if (pick < 0 || t < pick_t) {
        pick = i;
        pick_t = t;
      }
    }
    best = pick;
    best_slices = slices[best];
  }
  p->cand_chosen = best;
  if (best < 0)
    return fail(TNQ_ERR_PLAN_INFEASIBLE,
                "no contraction tree and slicing keeps every intermediate within 2^" +
                    std::to_string(o.max_intermediate_log2) + " elements");
  p->tree = cands[best];
  p->sliced.assign(h.n_labels, 0);
  p->slice_labels = best_slices;
  for (int l : best_slices) p->sliced[l] = 1;
  p->cost = tree_cost(h, p->tree, p->sliced);
  layout_steps(p);
  p->search_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return TNQ_OK;
}

}  // namespace tnq
