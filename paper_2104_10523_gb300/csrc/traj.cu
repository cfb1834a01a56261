// Kraus-trajectory sampler (builds trajectory leaves on the GPU) and the FP64
// reductions of noisy bitstring probabilities.  See traj.cuh.
#include <algorithm>

#include "traj.cuh"

namespace tnq {

namespace {

// SplitMix64 (Steele, Lea & Flood 2014): the i-th output of the generator
// started at `seed` is mix(seed + i * golden_gamma).
__device__ __forceinline__ double draw_uniform(uint64_t seed, uint64_t traj, uint64_t chan) {
  const uint64_t i = (traj << 32) + chan + 1;
  uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return double(z >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__global__ void traj_leaf_kernel(const TrajLeafDesc* __restrict__ leaves, int n_leaves,
                                 const TrajFactor* __restrict__ factors, const double2* __restrict__ mats,
                                 const double* __restrict__ cumq, char* ws, uint64_t seed, uint64_t traj_base,
                                 int traj_log2, const int8_t* __restrict__ picks, int n_sel, int64_t n_terms) {
  const long long T = 1ll << traj_log2;
  const long long total = (long long)n_leaves * T;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int leaf = int(idx / T);
    const long long tau = idx % T;
    const TrajLeafDesc L = leaves[leaf];
    const int ns = L.n_slots, D = 1 << ns;
    double2 M[16];
    for (int i = 0; i < 16; ++i) M[i] = make_double2(0.0, 0.0);
    for (int i = 0; i < D; ++i) M[i * D + i] = make_double2(1.0, 0.0);
    for (int f = 0; f < L.n_factors; ++f) {
      const TrajFactor F = factors[L.factor_off + f];
      int mi = F.mat_off;
      if (F.channel == 2 || (F.channel == 1 && picks)) {
        // pick table: per term (observables) or per distinct trajectory (noise)
        const int64_t term = int64_t(traj_base) + tau;
        mi += term < n_terms ? int(picks[term * n_sel + F.chan_index]) : 0;
      } else if (F.channel) {
        const double u = draw_uniform(seed, traj_base + uint64_t(tau), uint64_t(F.chan_index));
        int k = F.n_ops - 1;
        for (int j = 0; j < F.n_ops; ++j)
          if (u < cumq[F.cum_off + j]) {
            k = j;
            break;
          }
        mi += k;
      }
      const double2* U = mats + size_t(mi) * 16;
      double2 R[16];
      if (ns == 1) {  // 2x2 group, one-qubit op
        for (int r = 0; r < 2; ++r)
          for (int c = 0; c < 2; ++c)
            R[r * 2 + c] = cadd(cmul(U[r * 2 + 0], M[0 * 2 + c]), cmul(U[r * 2 + 1], M[1 * 2 + c]));
      } else if (F.arity == 2) {  // 4x4 op on both slots (indices swapped if listed reversed)
        for (int r = 0; r < 4; ++r)
          for (int c = 0; c < 4; ++c) {
            double2 s = make_double2(0.0, 0.0);
            for (int k2 = 0; k2 < 4; ++k2) {
              const int rr = F.swap ? (((r & 1) << 1) | (r >> 1)) : r;
              const int kk = F.swap ? (((k2 & 1) << 1) | (k2 >> 1)) : k2;
              s = cadd(s, cmul(U[rr * 4 + kk], M[k2 * 4 + c]));
            }
            R[r * 4 + c] = s;
          }
      } else {  // one-qubit op on slot 0 (most significant) or slot 1
        const int s0 = F.slot_mask == 1 ? 0 : 1;
        for (int r = 0; r < 4; ++r) {
          const int a = r >> 1, b = r & 1;
          for (int c = 0; c < 4; ++c) {
            double2 s;
            if (s0 == 0) s = cadd(cmul(U[a * 2 + 0], M[(0 << 1 | b) * 4 + c]), cmul(U[a * 2 + 1], M[(1 << 1 | b) * 4 + c]));
            else s = cadd(cmul(U[b * 2 + 0], M[(a << 1 | 0) * 4 + c]), cmul(U[b * 2 + 1], M[(a << 1 | 1) * 4 + c]));
            R[r * 4 + c] = s;
          }
        }
      }
      for (int i = 0; i < D * D; ++i) M[i] = R[i];
    }
    // write rows x free-input columns (closed inputs take column entry 0)
    const int rank_op = L.nfree + ns;
    float2* out = reinterpret_cast<float2*>(ws + L.out_offset) + (size_t(tau) << rank_op);
    for (int row = 0; row < D; ++row)
      for (int cf = 0; cf < (1 << L.nfree); ++cf) {
        int col = 0, bit = 0;
        for (int s = ns - 1; s >= 0; --s) {
          if ((L.in_fixed_mask >> s) & 1) continue;
          col |= ((cf >> bit) & 1) << (ns - 1 - s);
          ++bit;
        }
        const double2 v = M[row * D + col];
        out[(row << L.nfree) | cf] = make_float2(float(v.x), float(v.y));
      }
  }
}

struct Pos {
  int n;
  int p[32];
};

__device__ __forceinline__ size_t scatter(long long v, const Pos& P) {
  size_t r = 0;
  for (int j = 0; j < P.n; ++j)
    if ((v >> j) & 1) r |= size_t(1) << P.p[j];
  return r;
}

__global__ void noisy_accumulate_kernel(const double2* __restrict__ acc, int64_t nb, int64_t nt, Pos bp, Pos tp,
                                        double* psum, double* p2sum, const double* __restrict__ weights) {
  for (int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; b < nb; b += int64_t(gridDim.x) * blockDim.x) {
    const size_t base = scatter(b, bp);
    double s = 0.0, s2 = 0.0;
    for (int64_t t = 0; t < nt; ++t) {
      const double2 a = acc[base | scatter(t, tp)];
      const double p = a.x * a.x + a.y * a.y;
      const double w = weights ? weights[t] : 1.0;
      s += w * p;
      s2 += w * p * p;
    }
    psum[b] += s;
    p2sum[b] += s2;
  }
}

__global__ void noisy_finalize_kernel(const double* psum, const double* p2sum, int64_t nb, int64_t n, double* p,
                                      double* se) {
  for (int64_t b = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; b < nb; b += int64_t(gridDim.x) * blockDim.x) {
    const double m = psum[b] / double(n);
    p[b] = m;
    if (se) {
      const double var = fmax(p2sum[b] / double(n) - m * m, 0.0);
      se[b] = n > 1 ? sqrt(var / double(n - 1)) : 0.0;
    }
  }
}

__global__ void traj_amp_out_kernel(const double2* __restrict__ acc, int64_t nb, int64_t t0, int64_t nt, Pos bp,
                                    Pos tp, double2* out, int64_t stride) {
  const int64_t total = nb * nt;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t t = i / nb, b = i % nb;
    out[t * stride + b] = acc[scatter(b, bp) | scatter(t0 + t, tp)];
  }
}

Pos make_pos(const int* p, int n) {
  Pos P;
  P.n = n;
  for (int j = 0; j < n && j < 32; ++j) P.p[j] = p[j];
  return P;
}

unsigned blocks_for(int64_t n) { return unsigned(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096))); }

}  // namespace

cudaError_t launch_traj_leaves(const TrajLeafDesc* leaves, int n_leaves, const TrajFactor* factors,
                               const double2* mats, const double* cumq, char* ws, uint64_t seed,
                               uint64_t traj_base, int traj_log2, cudaStream_t st, const int8_t* picks, int n_sel,
                               int64_t n_terms) {
  if (n_leaves == 0) return cudaSuccess;
  const int64_t total = int64_t(n_leaves) << traj_log2;
  traj_leaf_kernel<<<blocks_for(total), 256, 0, st>>>(leaves, n_leaves, factors, mats, cumq, ws, seed, traj_base,
                                                      traj_log2, picks, n_sel, n_terms);
  return cudaGetLastError();
}

cudaError_t launch_noisy_accumulate(const void* acc, int64_t nb, int64_t nt, const int* bpos, int nbpos,
                                    const int* tpos, int ntpos, double* psum, double* p2sum, cudaStream_t st,
                                    const double* weights) {
  noisy_accumulate_kernel<<<blocks_for(nb), 256, 0, st>>>(reinterpret_cast<const double2*>(acc), nb, nt,
                                                          make_pos(bpos, nbpos), make_pos(tpos, ntpos), psum, p2sum,
                                                          weights);
  return cudaGetLastError();
}

cudaError_t launch_noisy_finalize(const double* psum, const double* p2sum, int64_t nb, int64_t n_traj, double* p,
                                  double* se, cudaStream_t st) {
  noisy_finalize_kernel<<<blocks_for(nb), 256, 0, st>>>(psum, p2sum, nb, n_traj, p, se);
  return cudaGetLastError();
}

cudaError_t launch_traj_amplitudes_out(const void* acc, int64_t nb, int64_t t0, int64_t nt, const int* bpos,
                                       int nbpos, const int* tpos, int ntpos, double2* out, int64_t out_stride,
                                       cudaStream_t st) {
  traj_amp_out_kernel<<<blocks_for(nb * nt), 256, 0, st>>>(reinterpret_cast<const double2*>(acc), nb, t0, nt,
                                                           make_pos(bpos, nbpos), make_pos(tpos, ntpos), out,
                                                           out_stride);
  return cudaGetLastError();
}

}  // namespace tnq
