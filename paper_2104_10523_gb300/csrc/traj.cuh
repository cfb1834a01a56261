// Kraus-trajectory leaf builder and the noisy-probability reductions.
//
// Stochastic noise (Sec. 3.3, Eq. kraus_sum): in trajectory t each channel c
// applies one Kraus operator A_k, drawn with probability q_k = Tr(A_k^dag A_k)/d
// and rescaled to A_k / sqrt(q_k), so the mean of |<x|psi_t>|^2 over
// trajectories is <x|rho|x>.  The draw for (t, c) is the (t * 2^32 + c + 1)-th
// output of a SplitMix64 generator started at the seed, turned into a double in
// [0, 1) from its top 53 bits; the pick is the first k with u < q_0 + ... + q_k.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tnq {

// One factor of a trajectory leaf's operator, in circuit order.
struct TrajFactor {
  int channel;     // 0: fixed gate matrix at mat_off; 1: Kraus channel; 2: operator
                   // selected per term from a pick table (Pauli observables)
  int arity;       // 1 or 2 (qubits the op acts on)
  int slot_mask;   // group slots the op acts on: 1, 2 or 3
  int swap;        // two-qubit op listed as (slot 1, slot 0)
  int mat_off;     // gate: index of its matrix; channel: index of A_0 / sqrt(q_0)
  int n_ops;       // channel: number of Kraus operators
  int cum_off;     // channel: index of q_0 in the cumulative-probability table
  int chan_index;  // channel: running channel index c in circuit order; selector: its column
                   // in the pick table
};

struct TrajLeafDesc {
  int n_slots;          // 1 or 2
  int in_fixed_mask;    // slot s input closed with |0> when bit s is set
  int n_factors;
  int factor_off;       // first TrajFactor of this leaf
  long long out_offset; // byte offset of the leaf tensor in the workspace
  int nfree;            // free input legs
};

// Builds every trajectory leaf for trajectories [traj_base, traj_base + 2^traj_log2).
// mats: complex128 matrices (row-major, 2x2 or 4x4) at the offsets the
// factors name (each matrix takes 16 entries); cumq: cumulative probabilities.
// Selector factors of trajectory (term) t use matrix mat_off + picks[t * n_sel
// + chan_index] (picks: device int8 [n_terms][n_sel]; terms t >= n_terms, the
// padding of a last pass, take pick 0).  With a pick table, Kraus channels
// take their pick from it as well (the distinct trajectories of a noisy
// estimate, drawn on the host) instead of drawing it.
cudaError_t launch_traj_leaves(const TrajLeafDesc* leaves, int n_leaves, const TrajFactor* factors,
                               const double2* mats, const double* cumq, char* ws, uint64_t seed,
                               uint64_t traj_base, int traj_log2, cudaStream_t st, const int8_t* picks = nullptr,
                               int n_sel = 0, int64_t n_terms = 0);

// For b < nb: psum[b] += sum_{t < nt} w_t |amp(b, t)|^2, p2sum[b] += sum_t w_t |amp|^4,
// with amp(b, t) = acc[pdep(b, bpos) | pdep(t, tpos)] (FP64, trajectories in
// order) and w_t = weights[t] (device; NULL: every weight 1).
cudaError_t launch_noisy_accumulate(const void* acc, int64_t nb, int64_t nt, const int* bpos, int nbpos,
                                    const int* tpos, int ntpos, double* psum, double* p2sum, cudaStream_t st,
                                    const double* weights = nullptr);

// p[b] = psum[b] / n, se[b] = sqrt(max(p2sum/n - p^2, 0) / (n - 1)) (se optional).
cudaError_t launch_noisy_finalize(const double* psum, const double* p2sum, int64_t nb, int64_t n_traj, double* p,
                                  double* se, cudaStream_t st);

// out[t * out_stride + b] = amp(b, t0 + t) for b < nb, t < nt (complex128).
cudaError_t launch_traj_amplitudes_out(const void* acc, int64_t nb, int64_t t0, int64_t nt, const int* bpos,
                                       int nbpos, const int* tpos, int ntpos, double2* out, int64_t out_stride,
                                       cudaStream_t st);

}  // namespace tnq
