// Internal data structures of the tensor-network amplitude engine.
//
// Host side: circuit -> grouped network (Sec. 3.1, Fig. 1; one- and two-qubit
// tensors merged as in Sec. 3.1.1, "small gate tensors are contracted
// internally to form larger tensors") -> hypergraph -> contraction tree
// (Sec. 3.1: FLOP minimisation by graph partitioning and heuristics) ->
// sliced indices (Sec. 3.1) -> per-step GEMM layouts.
// Device side: the executor runs every step as bit-permute + complex GEMM.
#pragma once

#include <complex>
#include <functional>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tnq.h"
#include "traj.cuh"

namespace tnq {

using cd = std::complex<double>;

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
tnq_status fail(tnq_status s, const std::string& msg);

// ---------------------------------------------------------------- circuit
struct COp {
  bool channel = false;
  std::vector<int> qubits;              // 1 or 2 qubits, qubits[0] = most significant
  std::vector<std::vector<cd>> mats;    // gate: 1 matrix; channel: Kraus operators
  std::vector<double> kraus_q;          // channel: q_k = Tr(A_k^dag A_k)/d
  int channel_index = -1;               // channel: running index in circuit order
  // selector (channel == true): one of mats is applied per term, chosen by a
  // pick table (the Pauli operators of an observable), without rescaling
  bool selector = false;
  int selector_index = -1;
};

struct Circuit {
  int n = 0;
  std::vector<COp> ops;
  int n_channels = 0;
  int n_selectors = 0;
};

// ---------------------------------------------------------------- network
enum LeafKind { LEAF_STATIC = 0, LEAF_PROJ = 1, LEAF_TRAJ = 2 };

// Product of a group of circuit ops acting on <= 2 qubits, as built on the GPU
// per trajectory for LEAF_TRAJ leaves.
struct GroupFactor {
  int op;        // index into Circuit::ops
  int slot_mask; // which group slots the op acts on: 1 = slot 0, 2 = slot 1, 3 = both
  bool swap;     // two-qubit op listed as (slot1, slot0)
};

struct Leaf {
  LeafKind kind = LEAF_STATIC;
  std::vector<int> labels;        // storage order: labels[p] names bit p
  std::vector<cd> data;           // LEAF_STATIC: 2^rank entries
  int qubit = -1;                 // LEAF_PROJ: the projected qubit
  // LEAF_TRAJ: operator on group slots, then legs fixed to |0>
  int n_slots = 0;                // 1 or 2
  std::vector<GroupFactor> factors;
  int in_fixed_mask = 0;          // slot s input leg fixed to |0> when bit s set
  int out_label[2] = {-1, -1};
  int in_label[2] = {-1, -1};
};

struct Network {
  int n_qubits = 0;
  int n_labels = 0;
  std::vector<Leaf> leaves;
  std::vector<char> is_output;    // per label: kept to the end (batch labels)
  std::vector<int> batch_labels;  // bit j of the bitstring index within a pass
  std::vector<int> traj_labels;   // bit j of the trajectory index within a pass
  // circuit wire of each label: qubit and position (position k = the qubit's
  // wire after its k-th op, 0 = the |0> input); -1 for batch/trajectory labels
  std::vector<int> label_qubit, label_pos;
  // open qubits (no projection; their final wires are output labels), in
  // increasing qubit order, and those output labels
  std::vector<int> open_qubits, open_labels;
  // projection leaf j reads entry proj_src[j] of a bitstring row of row_len
  // entries (row_len = n_qubits, or the register size of a doubled network)
  std::vector<int> proj_src;
  int row_len = 0;
  bool noisy = false;
};

// open: per qubit, 1 = leave its final wire open.  row_len: entries per
// bitstring row; projection leaf of qubit q reads entry q % row_len.
tnq_status build_network(const Circuit& c, int batch_log2, int traj_log2, const std::vector<char>& open, int row_len,
                         Network* out);

// ---------------------------------------------------------------- path search
struct Tree {
  int n_leaves = 0;
  std::vector<std::pair<int, int>> nodes;  // internal node i has id n_leaves + i (post order)
};

struct TreeCost {
  double flops = 0;      // one pass (one slice), 8 flops per complex MAC
  double bytes = 0;      // algorithmic bytes of one pass
  int max_log2 = 0;      // largest intermediate (log2 elements)
};

struct Hyper {
  int n_labels = 0;
  std::vector<std::vector<int>> leaf_labels;  // sorted
  std::vector<char> is_output;
  std::vector<int> label_count;
};

Hyper make_hyper(const Network& net);
TreeCost tree_cost(const Hyper& h, const Tree& t, const std::vector<char>& sliced);
Tree greedy_tree(const Hyper& h, const std::vector<char>& sliced, uint64_t seed, double temperature);
Tree bisect_tree(const Hyper& h, uint64_t seed, double imbalance, int leaf_group);
std::vector<int> choose_slices(const Hyper& h, const Tree& t, int cap_log2, bool* feasible);
// Local re-optimisation of t (sliced labels removed); returns the number of regions improved.
int reconfigure(const Hyper& h, Tree* t, const std::vector<char>& sliced, int cap_log2, int max_frontier, int sweeps);

// ---------------------------------------------------------------- plan
struct Step {
  int a = -1, b = -1, out = -1;   // tensor ids (leaves 0..L-1, then step outputs)
  int nH = 0, nM = 0, nN = 0, nK = 0;
  std::vector<int> a_req, b_req;  // required operand layouts: [K][M|N][H] (bit 0 first)
  std::vector<int> out_labels;    // [N][M][H]
  bool perm_a = false, perm_b = false;
  // no sliced label in the step's subtree: its result is the same for every
  // slice, so a batch computes it in its first slice only
  bool invariant = false;
  // subtree of static leaves only (no projection, trajectory or sliced index):
  // a constant of the circuit, contracted once when the plan is bound
  bool fold = false;
  // small slice-dependent subtree that keeps its sliced indices as batch
  // indices: one run per batch gives every slice's result at once, and the
  // per-slice steps that read it pick their slice like they do from a leaf
  bool sliced_batch = false;
  double flops = 0;
  // runs once per batch (in its first slice) rather than once per slice
  bool once() const { return invariant || sliced_batch; }
};

struct TensorSlot {
  std::vector<int> labels;        // effective labels (sliced removed), storage order for outputs
  int rank = 0;
  size_t offset = 0;              // byte offset in workspace
  bool leaf = false;
};

struct Plan {
  Network net;
  Hyper hyper;
  Tree tree;
  std::vector<char> sliced;       // per label
  std::vector<int> slice_labels;  // bit j of the slice id = value of slice_labels[j]
  std::vector<Step> steps;
  std::vector<TensorSlot> tensors;
  TreeCost cost;
  double search_ms = 0;
  int batch_log2 = 0, traj_log2 = 0;
  int cap_log2 = 31;              // max_intermediate_log2 the plan was made for
  int root = -1;
  // doubled density-matrix network (Sec. 3.3): results are the real numbers
  // <<x, x|rho>> = p(x), written as one double per bitstring
  bool density = false;
  // expectation values (Sec. 3.1.2): conjugate network with Pauli selectors;
  // picks[t * n_sel + j] = Pauli (0 I, 1 X, 2 Y, 3 Z) of term t on selector j
  bool expectation = false;
  int64_t n_terms = 0;
  int n_sel = 0;
  int kept_gates = 0;             // gates of the circuit inside the observable's light cone
  std::vector<int8_t> picks;
  size_t ws_picks = 0;
  // workspace layout (bytes)
  // persist: outputs of slice-invariant steps read by slice-dependent steps
  // (kept for the whole batch, outside the reusable arena)
  size_t ws_persist = 0, ws_persist_bytes = 0;
  size_t ws_leaves = 0, ws_arena = 0, ws_arena_bytes = 0, ws_scratch_a = 0, ws_scratch_b = 0, ws_partial = 0,
         ws_scratch_bytes = 0, ws_acc = 0, ws_misc = 0, ws_total = 0;
  // misc region: [flags 256 B][bit staging][output staging 16 B x 2^(w + n_open)][psum][p2sum]
  // [projection table: proj_src, then the row entries of the open qubits]
  size_t ws_bits = 0, ws_out_stage = 0, ws_psum = 0, ws_p2sum = 0, ws_qtab = 0;
  // trajectory program (noisy circuits): tables uploaded at bind time
  std::vector<TrajLeafDesc> traj_leaves;
  std::vector<int> traj_leaf_ids;
  std::vector<TrajFactor> traj_factors;
  std::vector<cd> traj_mats;      // 16 entries per matrix (2x2 use stride 2)
  std::vector<double> traj_cumq;
  size_t ws_traj = 0, ws_traj_factors = 0, ws_traj_mats = 0, ws_traj_cumq = 0;
  // cumulative Kraus probabilities per channel (by channel index), for the
  // host draws that find the distinct trajectories of an estimate, and the
  // workspace of one pass of distinct trajectories: picks [2^t][n_channels]
  // and their multiplicities [2^t]
  std::vector<std::vector<double>> chan_cumq;
  size_t ws_dedup_picks = 0, ws_dedup_w = 0;
  int64_t last_distinct = 0;      // distinct trajectories of the last noisy estimate
  uint64_t dedup_seed = 0;        // draws of the last estimate: seed, count, distinct picks
  int64_t dedup_n = -1;
  std::vector<int8_t> dedup_picks;
  std::vector<double> dedup_mult;
  int max_operand_log2 = 0;
  // candidate trees examined by the search: sliced flops per batch, predicted
  // time (learned ranking, else -1), the flop-minimal one and the chosen one
  std::vector<double> cand_flops, cand_pred;
  int cand_flopmin = -1, cand_chosen = -1;
  // autotuned kernel choice per step (for tuned_precision): -1 default rule,
  // 0 CUDA cores, 1 tensor cores
  std::vector<int8_t> kernel_choice;
  int tuned_precision = -1;
  // CUDA graph of one full batch (every slice and step), per precision
  void* graph_exec = nullptr;     // cudaGraphExec_t
  int graph_precision = -1;
  int graph_policy = -1;          // kernel policy the graph was captured with
  double graph_capture_ms = 0;
  int64_t graph_nodes = 0;
  // device binding
  void* bound_ws = nullptr;
  size_t bound_bytes = 0;
  int bound_precision = -1;
  // precision the folded (constant) steps were last contracted in; -1 = stale
  int folded_precision = -1;
};

// Shape of the network a plan contracts beyond the plain amplitude network:
// qubits left open (marginal wave-function slices) and the bitstring row
// length (a doubled network reads each row twice).
struct NetworkSpec {
  std::vector<char> open;
  int row_len = 0;
};

tnq_status make_plan(const Circuit& c, const tnq_plan_opts& o, Plan* p, const NetworkSpec& spec = NetworkSpec());
// A ranker returns the predicted time of one pass of a laid-out candidate plan.
using CandidateRanker = std::function<tnq_status(const Plan&, double*)>;
tnq_status make_plan_ranked(const Circuit& c, const tnq_plan_opts& o, Plan* p, const CandidateRanker* ranker,
                            const NetworkSpec& spec = NetworkSpec());
void layout_steps(Plan* p);

}  // namespace tnq

struct tnq_circuit { tnq::Circuit c; };
struct tnq_plan { tnq::Plan p; };
