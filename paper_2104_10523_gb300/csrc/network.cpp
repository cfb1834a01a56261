// Circuit -> tensor network (Sec. 3.1, Fig. 1) with projection leaves
// (Sec. 3.1.1, Fig. 2) and the internal merging of small gate tensors
// (Sec. 3.1.1: "small gate tensors are contracted internally to form larger
// tensors").
//
// Every two-qubit op seeds a group; each one-qubit op joins the next two-qubit
// group on its qubit (else the previous one, else a per-qubit chain group).  A
// group's tensor is the ordered product of its members; the input leg of the
// first group on a qubit is closed with |0>.  The last wire of qubit q ends in a
// projection leaf P_q[x_q, beta] = [bits(beta)[q] == x_q] whose batch labels
// beta enumerate the bitstrings of one pass, so one contraction yields the
// amplitudes of a whole batch.  Groups holding a Kraus channel become
// trajectory leaves: their data is built on the GPU per trajectory, and they
// carry the trajectory labels tau.
#include <algorithm>
#include <cmath>
#include <map>

#include "internal.h"

namespace tnq {

namespace {

// Embed a 1- or 2-qubit matrix into the group's slot space (dim 2^ns).
std::vector<cd> embed(const std::vector<cd>& U, int ns, int slot_mask, bool swap) {
  int D = 1 << ns;
  std::vector<cd> E(D * D, cd(0, 0));
  if (ns == 1) return U;  // single slot, single-qubit op
  if (slot_mask == 3) {
    if (!swap) return U;
    // U acts on (slot1, slot0): permute both row and column bit pairs.
    auto sw = [](int x) { return ((x & 1) << 1) | ((x >> 1) & 1); };
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) E[sw(r) * 4 + sw(c)] = U[r * 4 + c];
    return E;
  }
  // one-qubit op on slot s (slot 0 = most significant bit of the group index)
  int s = slot_mask == 1 ? 0 : 1;
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      int rb = s == 0 ? (r >> 1) : (r & 1);
      int cb = s == 0 ? (c >> 1) : (c & 1);
      int ro = s == 0 ? (r & 1) : (r >> 1);
      int co = s == 0 ? (c & 1) : (c >> 1);
      if (ro == co) E[r * 4 + c] = U[rb * 2 + cb];
    }
  return E;
}

std::vector<cd> matmul(const std::vector<cd>& A, const std::vector<cd>& B, int D) {
  std::vector<cd> C(D * D, cd(0, 0));
  for (int i = 0; i < D; ++i)
    for (int k = 0; k < D; ++k)
      for (int j = 0; j < D; ++j) C[i * D + j] += A[i * D + k] * B[k * D + j];
  return C;
}

// Contract two small static tensors over all shared labels (host, FP64).
// Result labels: a's remaining labels (in order) then b's.
void contract_host(const Leaf& a, const Leaf& b, Leaf* out) {
  std::vector<int> shared, ra, rb;
  for (int l : a.labels)
    if (std::find(b.labels.begin(), b.labels.end(), l) != b.labels.end()) shared.push_back(l);
    else ra.push_back(l);
  for (int l : b.labels)
    if (std::find(shared.begin(), shared.end(), l) == shared.end()) rb.push_back(l);
  out->labels = ra;
  out->labels.insert(out->labels.end(), rb.begin(), rb.end());
  int ro = (int)out->labels.size(), ks = (int)shared.size();
  out->data.assign(size_t(1) << ro, cd(0, 0));
  auto pos = [](const std::vector<int>& labs, int l) {
    return int(std::find(labs.begin(), labs.end(), l) - labs.begin());
  };
  for (size_t o = 0; o < (size_t(1) << ro); ++o) {
    size_t ia = 0, ib = 0;
    for (int p = 0; p < ro; ++p) {
      if (!((o >> p) & 1)) continue;
      int l = out->labels[p];
      if (p < (int)ra.size()) ia |= size_t(1) << pos(a.labels, l);
      else ib |= size_t(1) << pos(b.labels, l);
    }
    cd acc(0, 0);
    for (size_t k = 0; k < (size_t(1) << ks); ++k) {
      size_t ja = ia, jb = ib;
      for (int j = 0; j < ks; ++j)
        if ((k >> j) & 1) {
          ja |= size_t(1) << pos(a.labels, shared[j]);
          jb |= size_t(1) << pos(b.labels, shared[j]);
        }
      acc += a.data[ja] * b.data[jb];
    }
    out->data[o] = acc;
  }
}

}  // namespace

tnq_status build_network(const Circuit& c, int batch_log2, int traj_log2, const std::vector<char>& open, int row_len,
                         Network* out) {
  Network& net = *out;
  net = Network();
  net.n_qubits = c.n;
  net.row_len = row_len > 0 ? row_len : c.n;
  const int n = c.n;
  const int nops = (int)c.ops.size();
  net.noisy = c.n_channels > 0 || c.n_selectors > 0;

  // --- group assignment
  std::vector<int> group_of(nops, -1);
  std::vector<std::vector<int>> members;
  std::vector<std::vector<int>> gqubits;
  std::vector<std::vector<int>> twoq_on(n);
  for (int i = 0; i < nops; ++i)
    if (c.ops[i].qubits.size() == 2) {
      group_of[i] = (int)members.size();
      members.push_back({i});
      gqubits.push_back(c.ops[i].qubits);
      for (int q : c.ops[i].qubits) twoq_on[q].push_back(i);
    }
  std::vector<int> chain_group(n, -1);
  for (int i = 0; i < nops; ++i) {
    if (c.ops[i].qubits.size() != 1) continue;
    int q = c.ops[i].qubits[0];
    auto& v = twoq_on[q];
    auto it = std::upper_bound(v.begin(), v.end(), i);
    int g;
    if (it != v.end()) g = group_of[*it];
    else if (it != v.begin()) g = group_of[*(it - 1)];
    else {
      if (chain_group[q] < 0) {
        chain_group[q] = (int)members.size();
        members.push_back({});
        gqubits.push_back({q});
      }
      g = chain_group[q];
    }
    group_of[i] = g;
    members[g].push_back(i);
  }
  for (auto& m : members) std::sort(m.begin(), m.end());

  // --- groups in order along each qubit; wire labels
  // order key of a group on a qubit: its two-qubit seed's op index (chain: 0)
  std::vector<std::vector<int>> groups_on(n);
  for (int q = 0; q < n; ++q) {
    for (int i : twoq_on[q]) groups_on[q].push_back(group_of[i]);
    if (chain_group[q] >= 0) groups_on[q].push_back(chain_group[q]);
  }
  int next_label = 0;
  const int G = (int)members.size();
  std::vector<Leaf> gl(G);
  std::vector<int> final_label(n, -1);
  for (int g = 0; g < G; ++g) {
    gl[g].n_slots = (int)gqubits[g].size();
    gl[g].in_fixed_mask = 0;
  }
  auto new_label = [&](int q, int pos) {
    net.label_qubit.push_back(q);
    net.label_pos.push_back(pos);
    return next_label++;
  };
  for (int q = 0; q < n; ++q) {
    auto& gs = groups_on[q];
    int pos = 0;  // ops on q up to the current group boundary
    for (size_t j = 0; j < gs.size(); ++j) {
      int g = gs[j];
      for (int i : members[g])
        for (int qq : c.ops[i].qubits) pos += qq == q;
      int slot = gqubits[g][0] == q ? 0 : 1;
      if (j == 0) gl[g].in_fixed_mask |= 1 << slot;
      if (j + 1 < gs.size()) {
        int l = new_label(q, pos);
        gl[g].out_label[slot] = l;
        int g2 = gs[j + 1];
        int slot2 = gqubits[g2][0] == q ? 0 : 1;
        gl[g2].in_label[slot2] = l;
      } else {
        int l = new_label(q, pos);
        gl[g].out_label[slot] = l;
        final_label[q] = l;
      }
    }
  }

  // --- group tensors
  std::vector<Leaf> leaves;
  for (int g = 0; g < G; ++g) {
    Leaf& L = gl[g];
    int ns = L.n_slots, D = 1 << ns;
    bool has_channel = false;
    for (int i : members[g]) has_channel |= c.ops[i].channel;
    for (int i : members[g]) {
      GroupFactor f;
      f.op = i;
      const auto& qs = c.ops[i].qubits;
      if (qs.size() == 2) {
        f.slot_mask = 3;
        f.swap = qs[0] != gqubits[g][0];
      } else {
        f.slot_mask = (ns == 1 || qs[0] == gqubits[g][0]) ? 1 : 2;
        f.swap = false;
      }
      L.factors.push_back(f);
    }
    // storage labels: [free inputs (slot ns-1 .. 0)], [outputs (slot ns-1 .. 0)]
    L.labels.clear();
    for (int s = ns - 1; s >= 0; --s)
      if (!((L.in_fixed_mask >> s) & 1)) L.labels.push_back(L.in_label[s]);
    for (int s = ns - 1; s >= 0; --s) L.labels.push_back(L.out_label[s]);
    if (has_channel) {
      L.kind = LEAF_TRAJ;
    } else {
      L.kind = LEAF_STATIC;
      std::vector<cd> M(D * D, cd(0, 0));
      for (int d = 0; d < D; ++d) M[d * D + d] = 1;
      for (auto& f : L.factors) M = matmul(embed(c.ops[f.op].mats[0], ns, f.slot_mask, f.swap), M, D);
      // columns restricted to fixed inputs = 0
      int nfree = 0;
      for (int s = 0; s < ns; ++s) nfree += !((L.in_fixed_mask >> s) & 1);
      L.data.assign(size_t(D) << nfree, cd(0, 0));
      for (int row = 0; row < D; ++row)
        for (int cf = 0; cf < (1 << nfree); ++cf) {
          // map compact column (free slots, highest free slot most significant) to full column
          int col = 0, bit = 0;
          for (int s = ns - 1; s >= 0; --s) {
            if ((L.in_fixed_mask >> s) & 1) continue;
            int v = (cf >> bit) & 1;
            ++bit;
            col |= v << (ns - 1 - s);
          }
          L.data[(size_t(row) << nfree) | cf] = M[row * D + col];
        }
    }
    leaves.push_back(L);
  }
  // qubits without any op: |0> connected straight to the projection
  for (int q = 0; q < n; ++q)
    if (final_label[q] < 0) {
      Leaf L;
      L.kind = LEAF_STATIC;
      int l = new_label(q, 0);
      final_label[q] = l;
      L.labels = {l};
      L.data = {cd(1, 0), cd(0, 0)};
      leaves.push_back(L);
    }

  // --- merge small static tensors into static neighbours (host FP64)
  bool changed = true;
  while (changed) {
    changed = false;
    std::map<int, std::vector<int>> where;
    for (int i = 0; i < (int)leaves.size(); ++i)
      for (int l : leaves[i].labels) where[l].push_back(i);
    for (int i = 0; i < (int)leaves.size() && !changed; ++i) {
      if (leaves[i].kind != LEAF_STATIC || leaves[i].labels.size() > 2) continue;
      int best = -1;
      for (int l : leaves[i].labels)
        for (int j : where[l])
          if (j != i && leaves[j].kind == LEAF_STATIC &&
              (best < 0 || leaves[j].labels.size() > leaves[best].labels.size()))
            best = j;
      if (best < 0) continue;
      Leaf merged;
      merged.kind = LEAF_STATIC;
      contract_host(leaves[best], leaves[i], &merged);
      leaves[best] = merged;
      leaves.erase(leaves.begin() + i);
      changed = true;
    }
  }

  // --- batch and trajectory labels, projection leaves
  for (int j = 0; j < batch_log2; ++j) net.batch_labels.push_back(new_label(-1, -1));
  if (net.noisy)
    for (int j = 0; j < traj_log2; ++j) net.traj_labels.push_back(new_label(-1, -1));
  for (auto& L : leaves)
    if (L.kind == LEAF_TRAJ)
      for (int l : net.traj_labels) L.labels.push_back(l);
  for (int q = 0; q < n; ++q) {
    if (q < (int)open.size() && open[q]) {
      net.open_qubits.push_back(q);
      net.open_labels.push_back(final_label[q]);
      continue;
    }
    Leaf P;
    P.kind = LEAF_PROJ;
    P.qubit = q;
    P.labels = {final_label[q]};
    for (int l : net.batch_labels) P.labels.push_back(l);
    leaves.push_back(P);
    net.proj_src.push_back(q % net.row_len);
  }
  net.leaves = std::move(leaves);
  net.n_labels = next_label;
  net.is_output.assign(next_label, 0);
  for (int l : net.batch_labels) net.is_output[l] = 1;
  for (int l : net.traj_labels) net.is_output[l] = 1;
  for (int l : net.open_labels) net.is_output[l] = 1;
  return TNQ_OK;
}

}  // namespace tnq
