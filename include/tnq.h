/*
 * tnq.h -- C ABI of the GB300 tensor-network amplitude engine.
 *
 * The calls follow the problem statement of Sec. 3.1 of "Tensor Network
 * Quantum Virtual Machine for Simulating Quantum Circuits at Exascale"
 * (Nguyen et al., arXiv 2104.10523): a circuit goes in (Sec. 2.2, Sec. 3),
 * it is turned into a tensor network (Sec. 3.1, Fig. 1), a contraction path and
 * a set of sliced indices are found (Sec. 3.1), and the network is contracted
 * into bitstring amplitudes (Sec. 3.1.1, Eq. ampl_calc; the bit-string request
 * of Sec. 4.3) or, for circuits with Kraus channels (Sec. 3.3, Eq. kraus_sum),
 * into stochastic-trajectory estimates of bitstring probabilities.
 *
 * Conventions shared by every call:
 *   - all pointers are owned by the caller unless a call says otherwise;
 *     handles (tnq_circuit, tnq_plan, tnq_ctx) are owned by the library and
 *     released with the matching *_destroy call;
 *   - a buffer argument may be a host or a device pointer where the call
 *     says so; the library checks which with cudaPointerGetAttributes;
 *   - device memory: the library allocates none on its own; every byte it
 *     uses on the GPU lives in the workspace the caller binds to a plan;
 *   - calls never throw; on failure they return a status other than TNQ_OK
 *     and leave a message for tnq_last_error();
 *   - GPU calls are ordered on the context's stream and return after the
 *     results are complete (host outputs written, device outputs final).
 *
 * Layout conventions:
 *   - complex numbers are (re, im) pairs; double precision on the host side,
 *     complex64 (two floats) inside device tensors;
 *   - a k-qubit gate matrix is row-major 2^k x 2^k complex128, acting on the
 *     basis of its listed qubits with qubits[0] the most significant bit;
 *   - a bitstring is n int8 values bits[q] in {0,1} for qubit q;
 *   - a tensor whose indices all have dimension 2 is a flat array of 2^r
 *     complex64 entries; labels[p] names bit p of the flat index (bit 0 has
 *     stride 1).
 */
#ifndef TNQ_H
#define TNQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TNQ_OK = 0,
  TNQ_ERR_INVALID_ARG = 1,      /* bad qubit, non-unitary gate, incomplete Kraus set, bit not 0/1 */
  TNQ_ERR_PLAN_INFEASIBLE = 2,  /* no slicing meets max_intermediate_log2 */
  TNQ_ERR_WORKSPACE = 3,        /* bound workspace missing or too small */
  TNQ_ERR_CUDA = 4,             /* a CUDA runtime/driver call failed */
  TNQ_ERR_TIMEOUT = 5,          /* a bounded device-side wait expired */
  TNQ_ERR_NOT_SUPPORTED = 6,    /* mode or shape not available */
  TNQ_ERR_NO_DEVICE = 7         /* no usable sm_103 device */
} tnq_status;

/* Arithmetic of the pairwise-contraction GEMMs (Sec. 3.1 steps; TF32 as in the
 * paper's Table 2 A100 runs).  Storage is complex64 in every mode,
 * accumulation inside a GEMM is FP32, the cross-slice sums are FP64. */
typedef enum {
  TNQ_PREC_FP32 = 0,    /* CUDA-core FFMA complex GEMM, plain FP32 */
  TNQ_PREC_TF32 = 1,    /* tensor cores, one TF32 product */
  TNQ_PREC_TF32X3 = 2,  /* tensor cores, hi/lo TF32 split, 3 products */
  TNQ_PREC_BF16X3 = 3   /* tensor cores, hi/lo BF16 split, 3 products */
} tnq_precision;

/* How the contraction path is chosen (Sec. 3.1: FLOP minimisation by graph
 * partitioning and heuristics). */
typedef enum {
  TNQ_PATH_GREEDY = 0,  /* greedy pairwise, deterministic tie-break */
  TNQ_PATH_BISECT = 1,  /* recursive hypergraph bisection, best of n_candidates by FLOPs */
  TNQ_PATH_BEST = 2,    /* best by FLOPs over greedy and bisection candidates */
  TNQ_PATH_LEARNED = 3  /* candidates ranked by the learned cost model, if one is loaded */
} tnq_path_mode;

typedef struct tnq_circuit tnq_circuit;
typedef struct tnq_plan tnq_plan;
typedef struct tnq_ctx tnq_ctx;

typedef struct {
  int device;      /* CUDA device ordinal */
  void* stream;    /* cudaStream_t all work is ordered on; NULL = legacy default stream */
  int precision;   /* tnq_precision */
} tnq_options;

typedef struct {
  int max_intermediate_log2; /* cap on log2(elements) of any intermediate, batch bits
                                included; indices are sliced until it holds (Sec. 3.1) */
  int batch_log2;            /* bitstrings contracted together per pass: 2^batch_log2 */
  int traj_log2;             /* trajectories per pass for noisy circuits: 2^traj_log2 */
  int path_mode;             /* tnq_path_mode */
  int n_candidates;          /* candidate trees examined by BISECT/BEST/LEARNED */
  uint64_t seed;             /* seed of the randomised path search */
} tnq_plan_opts;

typedef struct {
  int n_leaves;              /* tensors after building and simplification (Sec. 3.1.1) */
  int n_steps;               /* pairwise contractions per pass */
  int n_sliced;              /* sliced indices; 2^n_sliced passes per batch */
  int max_log2;              /* largest intermediate, log2 elements, after slicing */
  int batch_log2, traj_log2;
  double flops_per_pass;     /* 8 real flops per complex multiply-add, one slice */
  double flops_per_batch;    /* flops executed per batch: steps whose subtree holds
                                no sliced label run once, the others once per slice */
  double bytes_per_pass;     /* algorithmic HBM bytes of the GEMM and permute steps */
  double search_ms;          /* host time of the path search and slicing */
  size_t workspace_bytes;    /* device bytes tnq_plan_bind needs */
  int n_open;                /* open qubits (tnq_plan_create_open); 0 otherwise */
  int64_t distinct_trajectories; /* distinct Kraus pick sequences the last
                                    tnq_noisy_probabilities call contracted */
} tnq_plan_info;

/* ---- library ---------------------------------------------------------- */
const char* tnq_version(void);
const char* tnq_status_string(tnq_status s);
/* Message of the last failed call on this thread (never NULL). */
const char* tnq_last_error(void);

/* ---- circuits (host only) ---------------------------------------------- */
/* A register of n_qubits qubits in |0...0> (Sec. 3.1: one rank-1 tensor per qubit).
 * Errors: INVALID_ARG if n_qubits < 1 or > 4096. */
tnq_status tnq_circuit_create(int n_qubits, tnq_circuit** out);
void tnq_circuit_destroy(tnq_circuit* c);
/* Append a 1- or 2-qubit gate (rank-2 / rank-4 tensor of Fig. 1a).
 * m: host, 2^arity x 2^arity complex128 row-major, copied.
 * Errors: INVALID_ARG for arity not 1 or 2, qubit out of range or repeated,
 * or a matrix with ||U^dagger U - I||_max > 1e-10. */
tnq_status tnq_circuit_gate(tnq_circuit* c, int arity, const int* qubits, const double* m);
/* Append a Kraus channel {A_k} (Eq. kraus_sum).  kraus: host, n_ops matrices of
 * 2^arity x 2^arity complex128, copied.  Errors: INVALID_ARG if n_ops < 1 or
 * > 64, or ||sum_k A_k^dagger A_k - I||_max > 1e-10. */
tnq_status tnq_circuit_channel(tnq_circuit* c, int arity, const int* qubits, int n_ops,
                               const double* kraus);
int tnq_circuit_n_qubits(const tnq_circuit* c);

/* ---- plans (host only) -------------------------------------------------- */
/* Build the projected tensor network of the circuit (Sec. 3.1, 3.1.1), absorb
 * one-qubit tensors into their neighbours, find a contraction tree and the
 * sliced indices (Sec. 3.1), and lay out every step.  No GPU work.
 * Errors: INVALID_ARG (bad options), PLAN_INFEASIBLE (cap cannot be met). */
tnq_status tnq_plan_create(const tnq_circuit* c, const tnq_plan_opts* opts, tnq_plan** out);
/* As tnq_plan_create, but the n_open listed qubits keep their final wires
 * open (Sec. 4.4, the marginal wave-function slice): their projections are
 * left out, so the network evaluates, per bitstring of the other qubits, to
 * the 2^n_open amplitudes <x_fixed, y| U |0...0> over all values y of the open
 * qubits.  tnq_amplitudes on such a plan expects -1 exactly at the open
 * qubits of every bitstring (the paper's marker of an open qubit) and returns
 * 2^n_open amplitudes per bitstring.  The open indices count towards
 * max_intermediate_log2 like the batch indices.  open_qubits: host, n_open
 * distinct qubit indices, copied.  Errors: INVALID_ARG (n_open outside
 * [0, 30], bad or repeated qubit), NOT_SUPPORTED (circuit with channels),
 * PLAN_INFEASIBLE as tnq_plan_create, also when batch_log2 + n_open exceeds
 * max_intermediate_log2. */
tnq_status tnq_plan_create_open(const tnq_circuit* c, const tnq_plan_opts* opts, int n_open, const int* open_qubits,
                                tnq_plan** out);
/* Exact noisy probabilities through the doubled density-matrix network of
 * Sec. 3.3 (Fig. 7a): the state |0><0| evolves as a tensor network on 2n
 * wires (ket wire q, bra wire q + n); a gate U acts as U on its ket wires and
 * conj(U) on its bra wires, and a one-qubit channel {A_k} (Eq. kraus_sum)
 * becomes the superoperator S = sum_k A_k (x) conj(A_k), a rank-4 tensor
 * joining the ket and bra wires of its qubit.  Closing both wires of every
 * qubit with <x_q| gives p(x) = <x|rho|x> (the trace of Fig. 7b with a
 * projector), evaluated with tnq_density_probabilities.  The plan finds a
 * path and slices for the doubled network as tnq_plan_create does (opts as
 * there; traj_log2 is ignored: nothing is sampled).  Errors: as
 * tnq_plan_create; NOT_SUPPORTED for a channel on two qubits; INVALID_ARG when
 * 2n exceeds 4096. */
tnq_status tnq_plan_create_density(const tnq_circuit* c, const tnq_plan_opts* opts, tnq_plan** out);
/* Expectation values <psi|H|psi> (Sec. 3.1.2, Eq. exp_val) of an observable
 * H = sum_t c_t P_t, P_t a product of Paulis, for |psi> = U|0...0>, by the
 * conjugate network of Fig. 3: the circuit's network, the Pauli tensors of a
 * term on the open legs, then the conjugate network, closed by <0...0|; the
 * value of that network is <0|U^dagger P_t U|0>.  Gates outside the backward
 * light cone of the observable's support cancel against their conjugates and
 * are left out (the simplification the paper notes for sparse observables).
 * The Pauli tensors of one qubit form an index over terms, so 2^traj_log2
 * terms are contracted together per pass, sharing the rest of the network.
 * paulis: host, [n_terms][n_qubits] chars from "IXYZ" (row t is term t,
 * entry q acts on qubit q), copied.  opts as tnq_plan_create; batch_log2 is
 * ignored, traj_log2 sets the terms per pass (at most those needed).
 * Errors: INVALID_ARG (n_terms outside [1, 2^24], another character),
 * NOT_SUPPORTED (circuit with channels), PLAN_INFEASIBLE as tnq_plan_create. */
tnq_status tnq_plan_create_expectation(const tnq_circuit* c, const tnq_plan_opts* opts, int64_t n_terms,
                                       const char* paulis, tnq_plan** out);
void tnq_plan_destroy(tnq_plan* p);
tnq_status tnq_plan_get_info(const tnq_plan* p, tnq_plan_info* info);
/* Per-step shape record: for step i, writes 8 ints
 * {a_rank, b_rank, out_rank, log2 H, log2 M, log2 N, log2 K,
 *  a_is_leaf | b_is_leaf << 1 | slice_invariant << 2}, where slice_invariant
 * marks a step whose subtree holds no sliced label (run once per batch).
 * rec must hold 8 * n_steps ints. */
tnq_status tnq_plan_get_steps(const tnq_plan* p, int* rec);

/* Contraction tree of a plan (Sec. 3.1: the sequence of pairwise
 * contractions), exported so that an independent contractor can follow the
 * same order.  pairs: [n_steps][2] ints, caller-owned; step i contracts the
 * tensors with ids pairs[2i] and pairs[2i+1], where ids 0 .. n_leaves-1 are the
 * plan's leaves and id n_leaves + j is the result of step j.  Sliced indices
 * are not part of the tree (slicing fixes indices, Sec. 3.1; the tree is the
 * same in every slice).  Errors: INVALID_ARG for NULL arguments. */
tnq_status tnq_plan_get_tree(const tnq_plan* p, int* pairs);
/* Indices of one leaf of a plan as circuit wires: wires[2j], wires[2j+1] =
 * (qubit, position) of the leaf's j-th index, where position k is the qubit's
 * wire right after the k-th op acting on it (0 = the |0> input; the last
 * position is the wire the bitstring projection closes, Sec. 3.1.1), and
 * (-1, -1) marks a batch or trajectory index.  A leaf is a group of circuit
 * ops merged into one tensor (Sec. 3.1.1), so its indices are the wires that
 * cross its boundary.  wires: caller-owned, 2 * max ints; copies min(max, *n)
 * entries and stores the leaf's rank in *n.
 * Errors: INVALID_ARG for a leaf outside [0, n_leaves) or NULL arguments. */
tnq_status tnq_plan_get_leaf_wires(const tnq_plan* p, int leaf, int max, int* wires, int* n);

/* ---- contexts and GPU execution ----------------------------------------- */
/* Errors: NO_DEVICE when the device is missing or not compute capability 10.3. */
tnq_status tnq_ctx_create(const tnq_options* opts, tnq_ctx** out);
void tnq_ctx_destroy(tnq_ctx* ctx);
tnq_status tnq_ctx_set_precision(tnq_ctx* ctx, int precision);

/* Bind a caller-owned device workspace of at least info.workspace_bytes to the
 * plan and upload its constant tensors into it.  The workspace must stay valid
 * and unused by others until the plan is destroyed or re-bound.
 * Errors: WORKSPACE if NULL or too small, CUDA. */
tnq_status tnq_plan_bind(tnq_ctx* ctx, tnq_plan* p, void* workspace, size_t bytes);

/* Amplitudes <x|U|0...0> (Eq. ampl_calc) for n_bs bitstrings.
 * bits: [n_bs][n_qubits] int8, host or device.  out: [n_bs][2] double (re, im),
 * host or device.  Bitstrings are processed 2^batch_log2 at a time, every
 * slice of a batch summed in FP64 in ascending slice order.
 * For a plan with open qubits (tnq_plan_create_open, Sec. 4.4) bits must hold
 * -1 exactly at the open qubits and out is [n_bs][2^n_open][2]: entry o of a
 * bitstring is the amplitude with the open qubits set to the bits of o, the
 * first open qubit (lowest index) the most significant bit of o.
 * Errors: INVALID_ARG (bit not 0/1, or not -1 at an open qubit; plan built
 * for a noisy circuit), WORKSPACE (plan not bound), CUDA. */
tnq_status tnq_amplitudes(tnq_ctx* ctx, tnq_plan* p, int64_t n_bs, const int8_t* bits,
                          double* out);

/* Partial amplitudes: as tnq_amplitudes, but only slices slice_begin ..
 * slice_begin + slice_count - 1 (of the plan's 2^n_sliced) are summed.  The
 * slices of Sec. 3.1 are independent sub-networks, so summing the partial
 * results of a partition of [0, 2^n_sliced) (in FP64, e.g. one block per GPU
 * followed by one all-reduce) gives the amplitudes.  Errors: INVALID_ARG for a
 * range outside [0, 2^n_sliced), otherwise as tnq_amplitudes. */
tnq_status tnq_amplitudes_slices(tnq_ctx* ctx, tnq_plan* p, int64_t n_bs, const int8_t* bits,
                                 int64_t slice_begin, int64_t slice_count, double* out);

/* Exact probabilities p(x) = <x|rho|x> of a density-matrix plan
 * (tnq_plan_create_density) for n_bs bitstrings of the circuit's n qubits.
 * bits: [n_bs][n] int8, host or device; p_out: [n_bs] double, host or device.
 * Bitstrings are processed 2^batch_log2 at a time; slices are summed in FP64
 * as for amplitudes.  p(x) is real; rounding leaves an imaginary part that is
 * dropped.  Errors: INVALID_ARG (not a density-matrix plan, bit not 0/1),
 * WORKSPACE, CUDA. */
tnq_status tnq_density_probabilities(tnq_ctx* ctx, tnq_plan* p, int64_t n_bs, const int8_t* bits, double* p_out);

/* Evaluate an expectation-value plan (tnq_plan_create_expectation):
 * *value = sum_t coeffs[t] * <psi|P_t|psi>, summed in FP64 in term order.
 * coeffs: host, [n_terms] real coefficients; term_values: host [n_terms] or
 * NULL, receives each <psi|P_t|psi> (real for Hermitian P_t; the rounding
 * imaginary part is dropped).  Errors: INVALID_ARG (not an expectation plan,
 * NULL coeffs or value), WORKSPACE, CUDA, TIMEOUT. */
tnq_status tnq_expectation(tnq_ctx* ctx, tnq_plan* p, const double* coeffs, double* value, double* term_values);

/* Noisy probabilities p(x) = <x|rho|x> estimated from n_traj stochastic
 * trajectories (Eq. kraus_sum channels, one Kraus operator drawn per channel
 * with probability Tr(A_k^dagger A_k)/d and rescaled by its inverse square
 * root, so the mean of |amp|^2 is unbiased).  Trajectory t, channel c draws
 * the (t*2^32 + c + 1)-th SplitMix64 output of `seed`.  The draws are made on
 * the host first; trajectories with the same picks on every channel have the
 * same amplitudes, so each distinct pick sequence is contracted once and
 * counted with its multiplicity (exact; tnq_plan_info reports how many were
 * distinct).
 * bits: [n_bs][n] int8 host or device; p_out, stderr_out: [n_bs] double, host
 * or device (stderr_out may be NULL).  Errors as tnq_amplitudes. */
tnq_status tnq_noisy_probabilities(tnq_ctx* ctx, tnq_plan* p, int64_t n_traj, uint64_t seed,
                                   int64_t n_bs, const int8_t* bits, double* p_out,
                                   double* stderr_out);

/* Amplitudes of individual trajectories (the unnormalised <x|psi_t> whose
 * squared moduli tnq_noisy_probabilities averages): trajectories
 * traj_begin .. traj_begin + n_traj - 1 with the same draws as above.
 * out: [n_traj][n_bs][2] double (re, im), host or device.  Errors as
 * tnq_noisy_probabilities. */
tnq_status tnq_trajectory_amplitudes(tnq_ctx* ctx, tnq_plan* p, uint64_t seed, int64_t traj_begin,
                                     int64_t n_traj, int64_t n_bs, const int8_t* bits, double* out);

/* One pairwise contraction (a single step of Sec. 3.1's sequence) of device
 * tensors A (rank ra, labels a_labels) and B (rank rb, labels b_labels) into
 * C (rank rc, labels c_labels): C = sum over the labels A and B share but C
 * lacks of A*B.  Labels shared by A, B and C are batch indices.  A, B, C:
 * device complex64.  workspace: device scratch of at least
 * tnq_contract_workspace_bytes(...) bytes.  Uses the context's precision.
 * Errors: INVALID_ARG (label sets inconsistent, rank > 31), WORKSPACE, CUDA. */
size_t tnq_contract_workspace_bytes(int precision, int ra, int rb, int rc);
tnq_status tnq_contract_pair(tnq_ctx* ctx, const void* A, int ra, const int* a_labels,
                             const void* B, int rb, const int* b_labels, void* C, int rc,
                             const int* c_labels, void* workspace, size_t workspace_bytes);

/* Pairwise contraction that allocates no device memory (the paper has no
 * counterpart).  Same operation, arguments and precision handling as
 * tnq_contract_pair, without the workspace: for callers that may not allocate
 * device memory while they run, such as programs whose own pool allocator owns
 * all device memory, or latency-critical loops that cannot accept the device
 * synchronisation that freeing memory implies.  Its scratch is one static
 * device array of 64 MiB inside the library.  With CUDA's lazy module loading
 * (the default) the array is committed on a device by the first call there,
 * which looks up its address, and it stays until the process exits; a caller
 * whose own pool takes all device memory must make that first call before
 * the pool reserves it, and the first call should come before any stream
 * capture.  A call returns after the contraction has completed (it
 * synchronizes the context's stream), and the context's per-kernel timing
 * records are not taken for it.  All calls share the array and it keeps the
 * last call's contents, so calls that overlap on the GPU race.  Errors:
 * INVALID_ARG when the contraction needs more than 64 MiB of scratch (see
 * tnq_contract_workspace_bytes) or the labels are inconsistent; TIMEOUT, CUDA
 * as tnq_contract_pair. */
tnq_status tnq_contract_pair_noalloc(tnq_ctx* ctx, const void* A, int ra, const int* a_labels, const void* B,
                                     int rb, const int* b_labels, void* C, int rc, const int* c_labels);

/* Autotune a bound plan for the context's precision: every step that could run
 * on the tensor cores is timed (CUDA events, best of `reps` after a warm-up run,
 * on the plan's workspace) both there and on the CUDA cores (row-streaming,
 * dot or tiled FP32 kernel); a tall-skinny step (one operand of at most 128
 * rows, K <= 256) is also timed with the large operand gathered, split and
 * multiplied in one tensor-core kernel.  The fastest choice is kept in the plan for
 * that precision; later calls at that precision follow it (and re-capture
 * their graph).  Results are unchanged in meaning (each choice meets the
 * precision's bound).  Optional outputs: steps placed on each kind of core. */
tnq_status tnq_plan_autotune(tnq_ctx* ctx, tnq_plan* p, int reps, int* n_tensor_core, int* n_cuda_core);

/* Replay full batches from a CUDA graph (1, the default) or launch every kernel
 * directly (0).  With graphs on, the first full batch of a plan at a given
 * precision captures every slice and step of one batch into a graph (on a
 * private stream) and later batches replay it on the context's stream.  The
 * results are identical either way.  Ragged last batches and timed runs
 * (tnq_ctx_set_timing) always launch directly. */
tnq_status tnq_ctx_set_graphs(tnq_ctx* ctx, int enable);

/* Which kernels run the steps of a plan.  TNQ_KERNELS_DEFAULT: the plan's
 * autotuned choice for the context's precision if it has one, else the
 * built-in rule (small, skinny and dot-shaped steps stay on the CUDA cores in
 * FP32, since they are launch- or bandwidth-bound).  TNQ_KERNELS_TENSOR_CORES:
 * in a tensor-core precision, every step that a tensor-core kernel accepts runs
 * there (the tall-skinny kernel where its shape rules hold, else the general
 * tensor-core GEMM); the others keep the built-in rule.  Results stay within
 * the precision's bound either way.  Errors: INVALID_ARG for another value. */
enum { TNQ_KERNELS_DEFAULT = 0, TNQ_KERNELS_TENSOR_CORES = 1 };
tnq_status tnq_ctx_set_kernel_policy(tnq_ctx* ctx, int policy);

/* ---- learned path cost model ----------------------------------------------- */
/* A 3-layer MLP (d_in -> hidden -> hidden -> 1, ReLU; BF16 weights with FP32
 * master copies and FP32 accumulation) that predicts ln(microseconds) of one
 * contraction step from its features, trained by Adam on MSE with the
 * library's own GPU kernels on step timings the contractor records
 * (tnq_ctx_get_timings).  A plan's predicted time is the sum of its steps'
 * exp(prediction) times its slice count.  The paper motivates ranking paths
 * by measured cost rather than FLOPs (Sec. 4.3: a path with more flops ran
 * more efficiently) but gives no model.
 * Parameters are one flat FP32 vector: W1 [d_in][hidden], b1 [hidden],
 * W2 [hidden][hidden], b2 [hidden], W3 [hidden][1], b3 [1]. */
typedef struct tnq_cost_model tnq_cost_model;
int tnq_step_feature_count(void);
/* d_in must equal tnq_step_feature_count(); weights He-uniform from `seed`. */
tnq_status tnq_cost_model_create(int d_in, int hidden, int max_batch, uint64_t seed, tnq_cost_model** out);
void tnq_cost_model_destroy(tnq_cost_model* m);
size_t tnq_cost_model_workspace_bytes(const tnq_cost_model* m);
int64_t tnq_cost_model_n_params(const tnq_cost_model* m);
/* Bind a caller-owned device workspace (weights, Adam state, activations). */
tnq_status tnq_cost_model_bind(tnq_ctx* ctx, tnq_cost_model* m, void* workspace, size_t bytes);
/* Host FP32 parameter vector in / out (set resets the Adam state). */
tnq_status tnq_cost_model_set_params(tnq_ctx* ctx, tnq_cost_model* m, const float* params);
tnq_status tnq_cost_model_get_params(tnq_ctx* ctx, tnq_cost_model* m, float* params);
/* One forward and backward pass on n <= max_batch host rows X [n][d_in] with
 * targets t [n]: gradients of the mean squared error (host, parameter layout)
 * and the loss.  grads or loss may be NULL. */
tnq_status tnq_cost_model_gradients(tnq_ctx* ctx, tnq_cost_model* m, const float* X, const float* t, int64_t n,
                                    float* grads, float* loss);
/* Adam training on host rows (seeded minibatch order per epoch). */
tnq_status tnq_cost_model_train(tnq_ctx* ctx, tnq_cost_model* m, const float* X, const float* t, int64_t n,
                                int epochs, int batch, float lr, float* final_loss);
/* Predictions y [n] for host rows X [n][d_in]. */
tnq_status tnq_cost_model_predict(tnq_ctx* ctx, tnq_cost_model* m, const float* X, int64_t n, float* y);
/* Features of every step of a plan for the kernels `precision` runs them on:
 * out [n_steps][tnq_step_feature_count()]. */
tnq_status tnq_plan_step_features(const tnq_plan* p, int precision, float* out);
/* As tnq_plan_create (BEST candidate set), but the candidate with the least
 * predicted time (at the context's precision) wins instead of the one with
 * the fewest flops. */
tnq_status tnq_plan_create_learned(tnq_ctx* ctx, tnq_cost_model* m, const tnq_circuit* c,
                                   const tnq_plan_opts* opts, tnq_plan** out);
/* Candidates the search examined: sliced flops per batch (-1 if infeasible)
 * and predicted milliseconds (-1 unless learned), the flop-minimal index and
 * the chosen index.  Copies min(max, *n) entries. */
tnq_status tnq_plan_get_candidates(const tnq_plan* p, double* flops, double* predicted_ms, int max, int* n,
                                   int* flopmin, int* chosen);

/* ---- measurement ---------------------------------------------------------- */
/* Number of kernels this context has launched so far (cumulative). */
tnq_status tnq_ctx_launch_count(const tnq_ctx* ctx, uint64_t* count);
/* Enable (1) or disable (0) per-kernel timing: every kernel the context
 * launches is bracketed by CUDA events on its stream, and one record per
 * launch is kept (enabling clears earlier records).  These per-step timings
 * (shape, algorithmic flops and bytes, duration) are also the training data
 * of the learned path cost model. */
tnq_status tnq_ctx_set_timing(tnq_ctx* ctx, int enable);
/* Copy up to max_records records, 10 doubles each:
 * {kind (0 permute, 1 CUDA-core GEMM, 2 tensor-core GEMM, 3 other), plan step,
 *  log2 H, log2 M, log2 N, log2 K, algorithmic flops, algorithmic bytes,
 *  milliseconds, 0}.  *n_out receives the number available. */
tnq_status tnq_ctx_get_timings(const tnq_ctx* ctx, double* rec, int max_records, int* n_out);

#ifdef __cplusplus
}
#endif
#endif /* TNQ_H */
