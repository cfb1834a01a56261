// extern "C" boundary (include/tnq.h).  Argument checking, handle ownership,
// error strings; the work happens in the planner and the executor.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "executor.h"
#include "internal.h"
#include "mlp.h"

namespace tnq {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

tnq_status fail(tnq_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

}  // namespace tnq

using namespace tnq;

namespace {

bool check_qubits(const Circuit& c, int arity, const int* qubits, std::string* why) {
  if (arity != 1 && arity != 2) {
    *why = "arity must be 1 or 2";
    return false;
  }
  if (!qubits) {
    *why = "qubits is NULL";
    return false;
  }
  for (int i = 0; i < arity; ++i)
    if (qubits[i] < 0 || qubits[i] >= c.n) {
      *why = "qubit index out of range";
      return false;
    }
  if (arity == 2 && qubits[0] == qubits[1]) {
    *why = "two-qubit op on a repeated qubit";
    return false;
  }
  return true;
}

std::vector<cd> read_matrix(const double* m, int d) {
  std::vector<cd> v(d * d);
  for (int i = 0; i < d * d; ++i) v[i] = cd(m[2 * i], m[2 * i + 1]);
  return v;
}

// max |(sum_k A_k^dag A_k) - I|
double completeness_error(const std::vector<std::vector<cd>>& mats, int d) {
  double worst = 0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      cd s(0, 0);
      for (auto& A : mats)
        for (int k = 0; k < d; ++k) s += std::conj(A[k * d + i]) * A[k * d + j];
      if (i == j) s -= 1.0;
      worst = std::max(worst, std::abs(s));
    }
  return worst;
}

}  // namespace

extern "C" {

const char* tnq_version(void) { return "tnq 0.1 (sm_103a)"; }

const char* tnq_status_string(tnq_status s) {
  switch (s) {
    case TNQ_OK: return "ok";
    case TNQ_ERR_INVALID_ARG: return "invalid argument";
    case TNQ_ERR_PLAN_INFEASIBLE: return "plan infeasible";
    case TNQ_ERR_WORKSPACE: return "workspace missing or too small";
    case TNQ_ERR_CUDA: return "CUDA error";
    case TNQ_ERR_TIMEOUT: return "device wait timed out";
    case TNQ_ERR_NOT_SUPPORTED: return "not supported";
    case TNQ_ERR_NO_DEVICE: return "no usable device";
  }
  return "unknown status";
}

const char* tnq_last_error(void) { return g_last_error.c_str(); }

tnq_status tnq_circuit_create(int n_qubits, tnq_circuit** out) {
  if (!out) return fail(TNQ_ERR_INVALID_ARG, "out is NULL");
  if (n_qubits < 1 || n_qubits > 4096) return fail(TNQ_ERR_INVALID_ARG, "n_qubits must be in [1, 4096]");
  auto* c = new (std::nothrow) tnq_circuit();
  if (!c) return fail(TNQ_ERR_INVALID_ARG, "out of host memory");
  c->c.n = n_qubits;
  *out = c;
  return TNQ_OK;
}

void tnq_circuit_destroy(tnq_circuit* c) { delete c; }

int tnq_circuit_n_qubits(const tnq_circuit* c) { return c ? c->c.n : 0; }

tnq_status tnq_circuit_gate(tnq_circuit* c, int arity, const int* qubits, const double* m) {
  if (!c || !m) return fail(TNQ_ERR_INVALID_ARG, "circuit or matrix is NULL");
  std::string why;
  if (!check_qubits(c->c, arity, qubits, &why)) return fail(TNQ_ERR_INVALID_ARG, why);
  int d = 1 << arity;
  COp op;
  op.qubits.assign(qubits, qubits + arity);
  op.mats.push_back(read_matrix(m, d));
  for (auto& z : op.mats[0])
    if (!std::isfinite(z.real()) || !std::isfinite(z.imag())) return fail(TNQ_ERR_INVALID_ARG, "non-finite gate");
  if (completeness_error(op.mats, d) > 1e-10) return fail(TNQ_ERR_INVALID_ARG, "gate matrix is not unitary");
  c->c.ops.push_back(std::move(op));
  return TNQ_OK;
}

tnq_status tnq_circuit_channel(tnq_circuit* c, int arity, const int* qubits, int n_ops, const double* kraus) {
  if (!c || !kraus) return fail(TNQ_ERR_INVALID_ARG, "circuit or Kraus array is NULL");
  std::string why;
  if (!check_qubits(c->c, arity, qubits, &why)) return fail(TNQ_ERR_INVALID_ARG, why);
  if (n_ops < 1 || n_ops > 64) return fail(TNQ_ERR_INVALID_ARG, "n_ops must be in [1, 64]");
  int d = 1 << arity;
  COp op;
  op.channel = true;
  op.qubits.assign(qubits, qubits + arity);
  for (int k = 0; k < n_ops; ++k) op.mats.push_back(read_matrix(kraus + 2 * size_t(k) * d * d, d));
  if (completeness_error(op.mats, d) > 1e-10)
    return fail(TNQ_ERR_INVALID_ARG, "Kraus operators do not satisfy sum A^dag A = I");
  for (auto& A : op.mats) {
    double q = 0;
    for (auto& z : A) q += std::norm(z);
    op.kraus_q.push_back(q / d);
  }
  op.channel_index = c->c.n_channels++;
  c->c.ops.push_back(std::move(op));
  return TNQ_OK;
}

tnq_status tnq_plan_create(const tnq_circuit* c, const tnq_plan_opts* opts, tnq_plan** out) {
  if (!c || !opts || !out) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  auto* p = new (std::nothrow) tnq_plan();
  if (!p) return fail(TNQ_ERR_INVALID_ARG, "out of host memory");
  tnq_status s = make_plan(c->c, *opts, &p->p);
  if (s != TNQ_OK) {
    delete p;
    return s;
  }
  *out = p;
  return TNQ_OK;
}

tnq_status tnq_plan_create_open(const tnq_circuit* c, const tnq_plan_opts* opts, int n_open, const int* open_qubits,
                                tnq_plan** out) {
  if (!c || !opts || !out || (n_open > 0 && !open_qubits)) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  if (n_open < 0 || n_open > 30) return fail(TNQ_ERR_INVALID_ARG, "n_open must be in [0, 30]");
  if (c->c.n_channels > 0) return fail(TNQ_ERR_NOT_SUPPORTED, "open qubits on a circuit with channels");
  NetworkSpec spec;
  spec.open.assign(c->c.n, 0);
  for (int i = 0; i < n_open; ++i) {
    const int q = open_qubits[i];
    if (q < 0 || q >= c->c.n) return fail(TNQ_ERR_INVALID_ARG, "open qubit out of range");
    if (spec.open[q]) return fail(TNQ_ERR_INVALID_ARG, "open qubit listed twice");
    spec.open[q] = 1;
  }
  if (opts->batch_log2 + n_open > opts->max_intermediate_log2)
    return fail(TNQ_ERR_PLAN_INFEASIBLE, "batch bits plus open qubits exceed max_intermediate_log2");
  auto* p = new (std::nothrow) tnq_plan();
  if (!p) return fail(TNQ_ERR_INVALID_ARG, "out of host memory");
  tnq_status s = make_plan(c->c, *opts, &p->p, spec);
  if (s != TNQ_OK) {
    delete p;
    return s;
  }
  *out = p;
  return TNQ_OK;
}

// Doubled circuit of Sec. 3.3 on 2n wires: ket wire q, bra wire q + n.  A gate
// U acts as U on the ket wires and conj(U) on the bra wires; a one-qubit
// channel {A_k} on q becomes the superoperator S = sum_k A_k (x) conj(A_k) on
// (q, q + n), S[(i i'), (j j')] = sum_k A_k[i][j] conj(A_k[i'][j']).  The state
// starts in |0...0>|0...0> (rho = |0><0|) and <<x, x| of the result is p(x).
static tnq_status doubled_circuit(const Circuit& c, Circuit* d) {
  const int n = c.n;
  d->n = 2 * n;
  d->ops.clear();
  d->n_channels = 0;
  for (const COp& op : c.ops) {
    if (!op.channel) {
      COp ket = op;
      COp bra = op;
      for (auto& z : bra.mats[0]) z = std::conj(z);
      for (auto& q : bra.qubits) q += n;
      d->ops.push_back(std::move(ket));
      d->ops.push_back(std::move(bra));
      continue;
    }
    if (op.qubits.size() != 1) return fail(TNQ_ERR_NOT_SUPPORTED, "two-qubit channels in a density-matrix network");
    std::vector<cd> S(16, cd(0, 0));
    for (const auto& A : op.mats)
      for (int i = 0; i < 2; ++i)
        for (int ip = 0; ip < 2; ++ip)
          for (int j = 0; j < 2; ++j)
            for (int jp = 0; jp < 2; ++jp) S[(i * 2 + ip) * 4 + (j * 2 + jp)] += A[i * 2 + j] * std::conj(A[ip * 2 + jp]);
    COp sup;
    sup.qubits = {op.qubits[0], op.qubits[0] + n};
    sup.mats = {S};
    d->ops.push_back(std::move(sup));
  }
  return TNQ_OK;
}

tnq_status tnq_plan_create_density(const tnq_circuit* c, const tnq_plan_opts* opts, tnq_plan** out) {
  if (!c || !opts || !out) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  if (2 * c->c.n > 4096) return fail(TNQ_ERR_INVALID_ARG, "doubled network exceeds 4096 wires");
  Circuit d;
  tnq_status s = doubled_circuit(c->c, &d);
  if (s != TNQ_OK) return s;
  auto* p = new (std::nothrow) tnq_plan();
  if (!p) return fail(TNQ_ERR_INVALID_ARG, "out of host memory");
  NetworkSpec spec;
  spec.row_len = c->c.n;
  tnq_plan_opts o = *opts;
  o.traj_log2 = 0;
  s = make_plan(d, o, &p->p, spec);
  if (s != TNQ_OK) {
    delete p;
    return s;
  }
  p->p.density = true;
  *out = p;
  return TNQ_OK;
}

tnq_status tnq_plan_create_expectation(const tnq_circuit* c, const tnq_plan_opts* opts, int64_t n_terms,
                                       const char* paulis, tnq_plan** out) {
  if (!c || !opts || !out || (n_terms > 0 && !paulis)) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  if (n_terms < 1 || n_terms > (int64_t(1) << 24)) return fail(TNQ_ERR_INVALID_ARG, "n_terms must be in [1, 2^24]");
  if (c->c.n_channels > 0) return fail(TNQ_ERR_NOT_SUPPORTED, "expectation values of a circuit with channels");
  const int n = c->c.n;
  // support of the observable: qubits where some term is not the identity
  std::vector<char> supp(n, 0);
  for (int64_t t = 0; t < n_terms; ++t)
    for (int q = 0; q < n; ++q) {
      const char ch = paulis[t * n + q];
      if (ch != 'I' && ch != 'X' && ch != 'Y' && ch != 'Z')
        return fail(TNQ_ERR_INVALID_ARG, "Pauli strings may hold only I, X, Y, Z");
      if (ch != 'I') supp[q] = 1;
    }
  // Light cone: U^dagger P U with a gate g of U that acts outside the support of
  // what follows it commutes past P and cancels against g^dagger.  Walking U
  // backwards, a gate is kept when it touches the current support, which it
  // then joins.
  std::vector<char> cone = supp;
  std::vector<char> keep(c->c.ops.size(), 0);
  for (int i = (int)c->c.ops.size() - 1; i >= 0; --i) {
    const COp& op = c->c.ops[i];
    bool touch = false;
    for (int q : op.qubits) touch |= cone[q] != 0;
    if (!touch) continue;
    keep[i] = 1;
    for (int q : op.qubits) cone[q] = 1;
  }
  Circuit d;
  d.n = n;
  int kept = 0;
  for (size_t i = 0; i < c->c.ops.size(); ++i)
    if (keep[i]) {
      d.ops.push_back(c->c.ops[i]);
      ++kept;
    }
  std::vector<int> sel_q;
  for (int q = 0; q < n; ++q)
    if (supp[q]) sel_q.push_back(q);
  const std::vector<cd> I2 = {cd(1, 0), cd(0, 0), cd(0, 0), cd(1, 0)}, X2 = {cd(0, 0), cd(1, 0), cd(1, 0), cd(0, 0)},
                        Y2 = {cd(0, 0), cd(0, -1), cd(0, 1), cd(0, 0)}, Z2 = {cd(1, 0), cd(0, 0), cd(0, 0), cd(-1, 0)};
  for (size_t j = 0; j < sel_q.size(); ++j) {
    COp op;
    op.channel = true;
    op.selector = true;
    op.selector_index = (int)j;
    op.qubits = {sel_q[j]};
    op.mats = {I2, X2, Y2, Z2};
    d.ops.push_back(std::move(op));
  }
  d.n_selectors = (int)sel_q.size();
  // the conjugate network: the kept gates' inverses in reverse order
  for (int i = (int)c->c.ops.size() - 1; i >= 0; --i) {
    if (!keep[i]) continue;
    COp inv = c->c.ops[i];
    const int D = 1 << (int)inv.qubits.size();
    std::vector<cd> m(D * D);
    for (int r = 0; r < D; ++r)
      for (int k = 0; k < D; ++k) m[r * D + k] = std::conj(inv.mats[0][k * D + r]);
    inv.mats[0] = m;
    d.ops.push_back(std::move(inv));
  }
  // qubits outside the light cone only contribute <0|0> = 1: renumber the
  // network's qubits to those that carry an op
  {
    std::vector<int> remap(n, -1);
    int m = 0;
    for (const COp& op : d.ops)
      for (int q : op.qubits)
        if (remap[q] < 0) remap[q] = 0;
    for (int q = 0; q < n; ++q)
      if (remap[q] == 0) remap[q] = m++;
    for (COp& op : d.ops)
      for (int& q : op.qubits) q = remap[q];
    d.n = std::max(m, 1);
  }
  auto* p = new (std::nothrow) tnq_plan();
  if (!p) return fail(TNQ_ERR_INVALID_ARG, "out of host memory");
  Plan& P = p->p;
  P.expectation = true;
  P.n_terms = n_terms;
  P.n_sel = (int)sel_q.size();
  P.kept_gates = kept;
  P.picks.resize(size_t(n_terms) * sel_q.size());
  for (int64_t t = 0; t < n_terms; ++t)
    for (size_t j = 0; j < sel_q.size(); ++j) {
      const char ch = paulis[t * n + sel_q[j]];
      P.picks[size_t(t) * sel_q.size() + j] = int8_t(ch == 'I' ? 0 : ch == 'X' ? 1 : ch == 'Y' ? 2 : 3);
    }
  tnq_plan_opts o = *opts;
  o.batch_log2 = 0;
  int need = 0;
  while ((int64_t(1) << need) < n_terms) ++need;
  o.traj_log2 = std::min(o.traj_log2, need);
  tnq_status s = make_plan(d, o, &P);
  if (s != TNQ_OK) {
    delete p;
    return s;
  }
  *out = p;
  return TNQ_OK;
}

tnq_status tnq_expectation(tnq_ctx* c, tnq_plan* p, const double* coeffs, double* value, double* term_values) {
  if (!c || !p) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  return exec_expectation(&c->c, &p->p, coeffs, value, term_values);
}

void tnq_plan_destroy(tnq_plan* p) {
  if (!p) return;
  plan_release_graph(&p->p);
  delete p;
}

tnq_status tnq_plan_get_info(const tnq_plan* pp, tnq_plan_info* info) {
  if (!pp || !info) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  const Plan& p = pp->p;
  info->n_leaves = (int)p.net.leaves.size();
  info->n_steps = (int)p.steps.size();
  info->n_sliced = (int)p.slice_labels.size();
  info->max_log2 = p.cost.max_log2;
  info->batch_log2 = p.batch_log2;
  info->traj_log2 = p.traj_log2;
  info->flops_per_pass = p.cost.flops;
  // executed flops: slice-invariant steps once per batch, the rest per slice
  const double n_slices = std::ldexp(1.0, (int)p.slice_labels.size());
  double fb = 0;
  for (const auto& s : p.steps) fb += s.fold ? 0.0 : s.once() ? s.flops : s.flops * n_slices;
  info->flops_per_batch = fb;
  info->bytes_per_pass = p.cost.bytes;
  info->search_ms = p.search_ms;
  info->workspace_bytes = p.ws_total;
  info->n_open = (int)p.net.open_qubits.size();
  info->distinct_trajectories = p.last_distinct;
  return TNQ_OK;
}

tnq_status tnq_plan_get_steps(const tnq_plan* pp, int* rec) {
  if (!pp || !rec) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  const Plan& p = pp->p;
  const int L = p.tree.n_leaves;
  for (size_t i = 0; i < p.steps.size(); ++i) {
    const Step& s = p.steps[i];
    int* r = rec + 8 * i;
    r[0] = (int)s.a_req.size();
    r[1] = (int)s.b_req.size();
    r[2] = (int)s.out_labels.size();
    r[3] = s.nH;
    r[4] = s.nM;
    r[5] = s.nN;
    r[6] = s.nK;
    r[7] = (s.a < L ? 1 : 0) | (s.b < L ? 2 : 0) | (s.invariant ? 4 : 0) | (s.fold ? 8 : 0) |
           (s.sliced_batch ? 16 : 0);
  }
  return TNQ_OK;
}

tnq_status tnq_plan_get_tree(const tnq_plan* pp, int* pairs) {
  if (!pp || !pairs) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  const Tree& t = pp->p.tree;
  for (size_t i = 0; i < t.nodes.size(); ++i) {
    pairs[2 * i] = t.nodes[i].first;
    pairs[2 * i + 1] = t.nodes[i].second;
  }
  return TNQ_OK;
}

tnq_status tnq_plan_get_leaf_wires(const tnq_plan* pp, int leaf, int max, int* wires, int* n) {
  if (!pp || !n || (max > 0 && !wires)) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  const Network& net = pp->p.net;
  if (leaf < 0 || leaf >= (int)net.leaves.size()) return fail(TNQ_ERR_INVALID_ARG, "leaf index out of range");
  const auto& labs = net.leaves[leaf].labels;
  *n = (int)labs.size();
  for (int j = 0; j < max && j < (int)labs.size(); ++j) {
    wires[2 * j] = net.label_qubit[labs[j]];
    wires[2 * j + 1] = net.label_pos[labs[j]];
  }
  return TNQ_OK;
}

tnq_status tnq_ctx_create(const tnq_options* o, tnq_ctx** out) {
  if (!o || !out) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  if (o->precision < TNQ_PREC_FP32 || o->precision > TNQ_PREC_BF16X3)
    return fail(TNQ_ERR_INVALID_ARG, "unknown precision");
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || o->device < 0 || o->device >= count) {
    cudaGetLastError();
    return fail(TNQ_ERR_NO_DEVICE, "no CUDA device with that ordinal");
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, o->device) != cudaSuccess) return fail(TNQ_ERR_NO_DEVICE, "device query failed");
  if (prop.major != 10 || prop.minor != 3)
    return fail(TNQ_ERR_NO_DEVICE, "this library is built for sm_103a (GB300) only");
  auto* c = new (std::nothrow) tnq_ctx();
  if (!c) return fail(TNQ_ERR_INVALID_ARG, "out of host memory");
  c->c.device = o->device;
  c->c.stream = static_cast<cudaStream_t>(o->stream);
  c->c.precision = o->precision;
  c->c.sm_count = prop.multiProcessorCount;
  *out = c;
  return TNQ_OK;
}

void tnq_ctx_destroy(tnq_ctx* c) {
  if (!c) return;
  for (auto e : c->c.ev_pool) cudaEventDestroy(e);
  if (c->c.capture_stream) cudaStreamDestroy(c->c.capture_stream);
  delete c;
}

tnq_status tnq_ctx_set_precision(tnq_ctx* c, int precision) {
  if (!c) return fail(TNQ_ERR_INVALID_ARG, "NULL context");
  if (precision < TNQ_PREC_FP32 || precision > TNQ_PREC_BF16X3) return fail(TNQ_ERR_INVALID_ARG, "unknown precision");
  c->c.precision = precision;
  return TNQ_OK;
}

tnq_status tnq_plan_bind(tnq_ctx* c, tnq_plan* p, void* ws, size_t bytes) {
  if (!c || !p) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  return exec_bind(&c->c, &p->p, ws, bytes);
}

tnq_status tnq_amplitudes(tnq_ctx* c, tnq_plan* p, int64_t n_bs, const int8_t* bits, double* out) {
  if (!c || !p) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  if (p->p.density) return fail(TNQ_ERR_INVALID_ARG, "density-matrix plan; use tnq_density_probabilities");
  return exec_amplitudes(&c->c, &p->p, n_bs, bits, out);
}

tnq_status tnq_density_probabilities(tnq_ctx* c, tnq_plan* p, int64_t n_bs, const int8_t* bits, double* p_out) {
  if (!c || !p) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  if (!p->p.density) return fail(TNQ_ERR_INVALID_ARG, "plan is not a density-matrix plan (tnq_plan_create_density)");
  return exec_amplitudes(&c->c, &p->p, n_bs, bits, p_out);
}

tnq_status tnq_amplitudes_slices(tnq_ctx* c, tnq_plan* p, int64_t n_bs, const int8_t* bits, int64_t slice_begin,
                                 int64_t slice_count, double* out) {
  if (!c || !p) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  if (p->p.density) return fail(TNQ_ERR_INVALID_ARG, "density-matrix plan; use tnq_density_probabilities");
  return exec_amplitudes_range(&c->c, &p->p, n_bs, bits, slice_begin, slice_count, out);
}

tnq_status tnq_noisy_probabilities(tnq_ctx* c, tnq_plan* p, int64_t n_traj, uint64_t seed, int64_t n_bs,
                                   const int8_t* bits, double* p_out, double* se_out) {
  if (!c || !p) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  return exec_noisy(&c->c, &p->p, n_traj, seed, n_bs, bits, p_out, se_out);
}

tnq_status tnq_trajectory_amplitudes(tnq_ctx* c, tnq_plan* p, uint64_t seed, int64_t traj_begin, int64_t n_traj,
                                     int64_t n_bs, const int8_t* bits, double* out) {
  if (!c || !p) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  return exec_traj_amplitudes(&c->c, &p->p, seed, traj_begin, n_traj, n_bs, bits, out);
}

size_t tnq_contract_workspace_bytes(int precision, int ra, int rb, int rc) {
  if (ra < 0 || rb < 0 || rc < 0 || ra > 31 || rb > 31 || rc > 31) return 0;
  return contract_workspace_bytes(precision, ra, rb, rc);
}

tnq_status tnq_contract_pair(tnq_ctx* c, const void* A, int ra, const int* al, const void* B, int rb,
                             const int* bl, void* C, int rc, const int* cl, void* ws, size_t ws_bytes) {
  if (!c || !A || !B || !C) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  if ((ra && !al) || (rb && !bl) || (rc && !cl)) return fail(TNQ_ERR_INVALID_ARG, "NULL label array");
  return exec_contract_pair(&c->c, A, ra, al, B, rb, bl, C, rc, cl, ws, ws_bytes);
}

// ---- learned path cost model
tnq_status tnq_cost_model_create(int d_in, int hidden, int max_batch, uint64_t seed, tnq_cost_model** out) {
  if (!out) return fail(TNQ_ERR_INVALID_ARG, "out is NULL");
  if (d_in != kStepFeatures) return fail(TNQ_ERR_INVALID_ARG, "d_in must equal tnq_step_feature_count()");
  if (hidden < 1 || hidden > 4096 || max_batch < 1 || max_batch > (1 << 20))
    return fail(TNQ_ERR_INVALID_ARG, "hidden must be in [1, 4096] and max_batch in [1, 2^20]");
  auto* m = new (std::nothrow) tnq_cost_model();
  if (!m) return fail(TNQ_ERR_INVALID_ARG, "out of host memory");
  m->m.d_in = d_in;
  m->m.h = hidden;
  m->m.max_batch = max_batch;
  m->m.seed = seed;
  m->m.layout();
  mlp_init(&m->m);
  *out = m;
  return TNQ_OK;
}

void tnq_cost_model_destroy(tnq_cost_model* m) { delete m; }

size_t tnq_cost_model_workspace_bytes(const tnq_cost_model* m) { return m ? m->m.ws_bytes : 0; }

int64_t tnq_cost_model_n_params(const tnq_cost_model* m) { return m ? (int64_t)m->m.n_params() : 0; }

int tnq_step_feature_count(void) { return kStepFeatures; }

tnq_status tnq_cost_model_bind(tnq_ctx* c, tnq_cost_model* m, void* ws, size_t bytes) {
  if (!c || !m) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  return mlp_bind(&c->c, &m->m, ws, bytes);
}

tnq_status tnq_cost_model_set_params(tnq_ctx* c, tnq_cost_model* m, const float* params) {
  if (!c || !m || !params) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  return mlp_upload(&c->c, &m->m, params);
}

tnq_status tnq_cost_model_get_params(tnq_ctx* c, tnq_cost_model* m, float* params) {
  if (!c || !m || !params) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  return mlp_download(&c->c, &m->m, params);
}

tnq_status tnq_cost_model_gradients(tnq_ctx* c, tnq_cost_model* m, const float* X, const float* t, int64_t n,
                                    float* grads, float* loss) {
  if (!c || !m || !X || !t) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  return mlp_gradients(&c->c, &m->m, X, t, n, grads, loss);
}

tnq_status tnq_cost_model_train(tnq_ctx* c, tnq_cost_model* m, const float* X, const float* t, int64_t n, int epochs,
                                int batch, float lr, float* final_loss) {
  if (!c || !m || !X || !t) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  return mlp_train(&c->c, &m->m, X, t, n, epochs, batch, lr, final_loss);
}

tnq_status tnq_cost_model_predict(tnq_ctx* c, tnq_cost_model* m, const float* X, int64_t n, float* y) {
  if (!c || !m || !X || !y) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  if (n < 0) return fail(TNQ_ERR_INVALID_ARG, "n must be >= 0");
  return mlp_predict(&c->c, &m->m, X, n, y);
}

tnq_status tnq_plan_step_features(const tnq_plan* p, int precision, float* out) {
  if (!p || !out) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  std::vector<float> f;
  step_features(p->p, precision, &f);
  std::copy(f.begin(), f.end(), out);
  return TNQ_OK;
}

tnq_status tnq_plan_create_learned(tnq_ctx* c, tnq_cost_model* m, const tnq_circuit* circ, const tnq_plan_opts* o,
                                   tnq_plan** out) {
  if (!c || !m || !circ || !o || !out) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  if (!m->m.ws) return fail(TNQ_ERR_WORKSPACE, "cost model has no bound workspace");
  auto* p = new (std::nothrow) tnq_plan();
  if (!p) return fail(TNQ_ERR_INVALID_ARG, "out of host memory");
  Ctx* ctx = &c->c;
  CostModel* cm = &m->m;
  // predicted pass time = sum over steps of exp(model(features)) (the model predicts ln microseconds)
  CandidateRanker rank = [ctx, cm](const Plan& cand, double* t) -> tnq_status {
    std::vector<float> f;
    step_features(cand, ctx->precision, &f);
    const int64_t n = int64_t(f.size()) / kStepFeatures;
    std::vector<float> y(n);
    tnq_status s = mlp_predict(ctx, cm, f.data(), n, y.data());
    if (s != TNQ_OK) return s;
    // a step's runs per batch: none when folded at bind, one when it runs
    // once per batch, one per slice otherwise; per slice on average
    const double ns = std::ldexp(1.0, (int)cand.slice_labels.size());
    double sum = 0;
    for (int64_t i = 0; i < n; ++i) {
      const Step& s = cand.steps[size_t(i)];
      const double runs = s.fold ? 0.0 : s.once() ? 1.0 : ns;
      sum += runs / ns * std::exp(double(y[size_t(i)]));
    }
    *t = sum * 1e-3;  // milliseconds per slice (the caller scales by the slice count)
    return TNQ_OK;
  };
  tnq_plan_opts o2 = *o;
  if (o2.path_mode == TNQ_PATH_GREEDY) o2.path_mode = TNQ_PATH_BEST;
  tnq_status s = make_plan_ranked(circ->c, o2, &p->p, &rank);
  if (s != TNQ_OK) {
    delete p;
    return s;
  }
  *out = p;
  return TNQ_OK;
}

tnq_status tnq_plan_get_candidates(const tnq_plan* pp, double* flops, double* predicted_ms, int max, int* n,
                                   int* flopmin, int* chosen) {
  if (!pp || !n) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  const Plan& p = pp->p;
  *n = (int)p.cand_flops.size();
  for (int i = 0; i < max && i < *n; ++i) {
    if (flops) flops[i] = p.cand_flops[i];
    if (predicted_ms) predicted_ms[i] = p.cand_pred[i];
  }
  if (flopmin) *flopmin = p.cand_flopmin;
  if (chosen) *chosen = p.cand_chosen;
  return TNQ_OK;
}

tnq_status tnq_plan_autotune(tnq_ctx* c, tnq_plan* p, int reps, int* n_tensor_core, int* n_cuda_core) {
  if (!c || !p) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  if (reps < 1 || reps > 100) return fail(TNQ_ERR_INVALID_ARG, "reps must be in [1, 100]");
  return exec_autotune(&c->c, &p->p, reps, n_tensor_core, n_cuda_core);
}

tnq_status tnq_ctx_set_graphs(tnq_ctx* c, int enable) {
  if (!c) return fail(TNQ_ERR_INVALID_ARG, "NULL context");
  c->c.use_graphs = enable != 0;
  return TNQ_OK;
}

tnq_status tnq_ctx_set_kernel_policy(tnq_ctx* c, int policy) {
  if (!c) return fail(TNQ_ERR_INVALID_ARG, "NULL context");
  if (policy != TNQ_KERNELS_DEFAULT && policy != TNQ_KERNELS_TENSOR_CORES)
    return fail(TNQ_ERR_INVALID_ARG, "unknown kernel policy");
  c->c.kernel_policy = policy;
  return TNQ_OK;
}

tnq_status tnq_ctx_launch_count(const tnq_ctx* c, uint64_t* count) {
  if (!c || !count) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  *count = c->c.launches;
  return TNQ_OK;
}

tnq_status tnq_ctx_set_timing(tnq_ctx* c, int enable) {
  if (!c) return fail(TNQ_ERR_INVALID_ARG, "NULL context");
  c->c.timing = enable != 0;
  if (enable) {
    c->c.records.clear();
    c->c.pending.clear();
  }
  return TNQ_OK;
}

tnq_status tnq_ctx_get_timings(const tnq_ctx* c, double* rec, int max_records, int* n_out) {
  if (!c || !n_out || (max_records > 0 && !rec)) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  const auto& R = c->c.records;
  *n_out = (int)R.size();
  for (int i = 0; i < max_records && i < (int)R.size(); ++i) {
    double* r = rec + 10 * size_t(i);
    r[0] = R[i].kind;
    r[1] = R[i].step;
    r[2] = R[i].nH;
    r[3] = R[i].nM;
    r[4] = R[i].nN;
    r[5] = R[i].nK;
    r[6] = R[i].flops;
    r[7] = R[i].bytes;
    r[8] = R[i].ms;
    r[9] = 0;
  }
  return TNQ_OK;
}

}  // extern "C"
