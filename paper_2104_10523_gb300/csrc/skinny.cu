// Bandwidth-oriented complex GEMMs for skinny contraction steps.
//
// Many steps of a contraction path have a tiny side: few output rows (a small
// operand meeting a large one) or a tiny output with a long contracted
// dimension (the inner products that close a network).  Their cost is reading
// the large operand once; a tiled GEMM would leave most lanes idle.
//
//   rows kernel:  C[h][s][g] = sum_k S[h][s][k] G[h][g][k] for a small side of
//                 at most 32 rows: each thread owns one row g of the large
//                 operand, the small operand and a K slice of G are staged in
//                 shared memory by coalesced loads; output strides make the
//                 same kernel serve both "small M" and "small N".
//   rows kernel, short K (<= 32): each thread loads its row of the large operand
//                 into registers with 16-byte loads (no staging);
//   dot kernel:   M, N <= 8 and long K: every thread walks its own part of K
//                 with 16-byte loads and keeps the M x N sums in registers; the
//                 CTA reduces them and writes one partial per CTA.
#include <algorithm>

#include "kernels.cuh"

namespace tnq {

namespace {

constexpr int RW_THREADS = 128;  // rows of the large operand per CTA
constexpr int RW_KC = 32;        // K elements staged per iteration
constexpr int RW_SMAX = 32;

__global__ void __launch_bounds__(RW_THREADS) cgemm_rows_kernel(
    const float2* __restrict__ S, const float2* __restrict__ G, float2* __restrict__ C, double2* __restrict__ acc,
    float2* __restrict__ part, int ns, int ng, int K, int batch, long long s_stride_out, long long g_stride_out,
    int kchunk, int tiles_g) {
  __shared__ float2 Gs[RW_THREADS][RW_KC + 1];
  __shared__ float2 Ss[RW_SMAX][RW_KC + 1];
  const int t = threadIdx.x;
  const int tile = int(blockIdx.x % tiles_g);
  const int h = int(blockIdx.x / tiles_g);
  const int g0 = tile * RW_THREADS;
  const int split = blockIdx.y;
  const int kbeg = split * kchunk, kend = min(K, kbeg + kchunk);
  const float2* Sh = S + size_t(h) * ns * K;
  const float2* Gh = G + size_t(h) * ng * K;
  float ar[RW_SMAX], ai[RW_SMAX];
#pragma unroll
  for (int s = 0; s < RW_SMAX; ++s) ar[s] = ai[s] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += RW_KC) {
    const int kc = min(RW_KC, kend - k0);
    // stage G[g0 .. g0+127][k0 .. k0+kc): row segments are contiguous in K
    for (int idx = t; idx < RW_THREADS * RW_KC; idx += RW_THREADS) {
      const int r = idx / RW_KC, kk = idx % RW_KC;
      float2 v = make_float2(0.f, 0.f);
      if (g0 + r < ng && kk < kc) v = Gh[size_t(g0 + r) * K + k0 + kk];
      Gs[r][kk] = v;
    }
    for (int idx = t; idx < RW_SMAX * RW_KC; idx += RW_THREADS) {
      const int r = idx / RW_KC, kk = idx % RW_KC;
      float2 v = make_float2(0.f, 0.f);
      if (r < ns && kk < kc) v = Sh[size_t(r) * K + k0 + kk];
      Ss[r][kk] = v;
    }
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
      const float2 g = Gs[t][kk];
#pragma unroll
      for (int s = 0; s < RW_SMAX; ++s) {
        if (s < ns) {
          const float2 a = Ss[s][kk];
          ar[s] = fmaf(a.x, g.x, ar[s]);
          ar[s] = fmaf(-a.y, g.y, ar[s]);
          ai[s] = fmaf(a.x, g.y, ai[s]);
          ai[s] = fmaf(a.y, g.x, ai[s]);
        }
      }
    }
    __syncthreads();
  }
  const int g = g0 + t;
  if (g >= ng) return;
  const size_t hbase = size_t(h) * ns * ng;
#pragma unroll
  for (int s = 0; s < RW_SMAX; ++s) {
    if (s < ns) {
      const size_t o = hbase + size_t(s) * s_stride_out + size_t(g) * g_stride_out;
      if (part) {
        part[size_t(split) * batch * ns * ng + o] = make_float2(ar[s], ai[s]);
      } else if (acc) {
        double2 v = acc[o];
        v.x += ar[s];
        v.y += ai[s];
        acc[o] = v;
      } else {
        C[o] = make_float2(ar[s], ai[s]);
      }
    }
  }
}

constexpr int DOT_THREADS = 256;

// Dot products for M, N <= 8: the M x N outputs form (M / TM) x (N / TN) <= 4
// blocks of TM x TN (TM = min(M, 4), TN = min(N, 4)); the block index sits in
// the low bits of the thread index, so the lanes of one warp that share a row
// read it in the same 16-byte load instruction and every loaded value serves
// TN (or TM) complex multiply-adds from registers.  Each thread keeps two
// K-pairs in flight per iteration; per-CTA partials go to part[split][batch][M][N].
//
// Each operand is addressed as row base + K offset, both bit deposits of the
// row index (row bits, then batch bits) and of k into the operand's stored bit
// positions (DotOp): a contiguous [batch][rows][K] operand has K in the low
// bits; an operand read in place (its permute fused) has them where it stores
// them, in increasing positions.  A thread advances its K offset by adding in
// the deposited domain: dep(k + d) = ((dep(k) | ~mask) + dep(d)) & mask, the
// carries running through the non-K positions.
__device__ __forceinline__ size_t dot_dep(long long v, const signed char* pos, int n) {
  size_t o = 0;
  for (int j = 0; j < n; ++j)
    if ((v >> j) & 1) o |= size_t(1) << pos[j];
  return o;
}

__device__ __forceinline__ size_t dep_add(size_t x, size_t inc, size_t mask) { return ((x | ~mask) + inc) & mask; }

template <int R>
__device__ __forceinline__ void cdot_load(const float2* __restrict__ p, const size_t (&row)[R], size_t koff, bool in,
                                          float4 (&v)[R]) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (in) v[i] = *reinterpret_cast<const float4*>(p + row[i] + koff);
  }
}

template <int TM, int TN>
__device__ __forceinline__ void cdot_fma(const float4 (&a)[TM], const float4 (&b)[TN], float (&cr)[TM][TN],
                                         float (&ci)[TM][TN]) {
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      cr[i][j] = fmaf(a[i].x, b[j].x, cr[i][j]);
      cr[i][j] = fmaf(-a[i].y, b[j].y, cr[i][j]);
      ci[i][j] = fmaf(a[i].x, b[j].y, ci[i][j]);
      ci[i][j] = fmaf(a[i].y, b[j].x, ci[i][j]);
      cr[i][j] = fmaf(a[i].z, b[j].z, cr[i][j]);
      cr[i][j] = fmaf(-a[i].w, b[j].w, cr[i][j]);
      ci[i][j] = fmaf(a[i].z, b[j].w, ci[i][j]);
      ci[i][j] = fmaf(a[i].w, b[j].z, ci[i][j]);
    }
}

template <int TM, int TN>
__global__ void __launch_bounds__(DOT_THREADS, 2) cdot_blk_kernel(const __grid_constant__ DotOp A,
                                                                  const __grid_constant__ DotOp B,
                                                                  float2* __restrict__ part, int M, int N, int K,
                                                                  int kchunk) {
  __shared__ float red[DOT_THREADS / 32][2 * 64];
  const int split = blockIdx.x, h = blockIdx.y;
  const int kbeg = split * kchunk, kend = min(K, kbeg + kchunk);
  const int nbj = N / TN, nb = (M / TM) * nbj;  // nb in {1, 2, 4}
  const int blk = threadIdx.x & (nb - 1), kq = threadIdx.x / nb;
  const int bi = blk / nbj, bj = blk % nbj;
  const int step = 2 * (DOT_THREADS / nb);  // K values one CTA iteration covers
  size_t ra[TM], rb[TN];
#pragma unroll
  for (int i = 0; i < TM; ++i) ra[i] = dot_dep((long long)h * M + bi * TM + i, A.rowpos, A.nrow);
#pragma unroll
  for (int j = 0; j < TN; ++j) rb[j] = dot_dep((long long)h * N + bj * TN + j, B.rowpos, B.nrow);
  const size_t ma = A.kmask, mb = B.kmask;
  const size_t a_step = dot_dep(step, A.kpos, A.nk), b_step = dot_dep(step, B.kpos, B.nk);
  const size_t a_2step = dot_dep(2 * step, A.kpos, A.nk), b_2step = dot_dep(2 * step, B.kpos, B.nk);
  float cr[TM][TN], ci[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) cr[i][j] = ci[i][j] = 0.f;
  // k is even and K bit 0 is stored bit 0 of both operands, so (k, k+1) is one
  // aligned 16-byte pair; kend is even
  int k = kbeg + 2 * kq;
  size_t ka = dot_dep(k, A.kpos, A.nk), kb = dot_dep(k, B.kpos, B.nk);
  for (; k < kend; k += 2 * step) {
    float4 a0[TM], b0[TN], a1[TM], b1[TN];
    const bool in1 = k + step < kend;
    cdot_load<TM>(A.p, ra, ka, true, a0);
    cdot_load<TN>(B.p, rb, kb, true, b0);
    cdot_load<TM>(A.p, ra, dep_add(ka, a_step, ma), in1, a1);
    cdot_load<TN>(B.p, rb, dep_add(kb, b_step, mb), in1, b1);
    cdot_fma<TM, TN>(a0, b0, cr, ci);
    cdot_fma<TM, TN>(a1, b1, cr, ci);
    ka = dep_add(ka, a_2step, ma);
    kb = dep_add(kb, b_2step, mb);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      float r = cr[i][j], im = ci[i][j];
      // sum over the lanes of the same block (lane bits above the block bits)
      for (int off = 16; off >= nb; off >>= 1) {
        r += __shfl_xor_sync(0xffffffffu, r, off);
        im += __shfl_xor_sync(0xffffffffu, im, off);
      }
      if (lane < nb) {
        red[warp][2 * (lane * TM * TN + i * TN + j)] = r;
        red[warp][2 * (lane * TM * TN + i * TN + j) + 1] = im;
      }
    }
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * M * N; q += DOT_THREADS) {
    float v = 0.f;
    for (int w = 0; w < DOT_THREADS / 32; ++w) v += red[w][q];
    const int b = q / (2 * TM * TN), ij = (q % (2 * TM * TN)) >> 1;
    const int i = (b / nbj) * TM + ij / TN, j = (b % nbj) * TN + ij % TN;
    float* dst = reinterpret_cast<float*>(part + (size_t(split) * gridDim.y + h) * M * N + size_t(i) * N + j);
    dst[q & 1] = v;
  }
}

// Small operand of ns <= 32 rows and K <= 32: each thread owns one row of the
// large operand and reads it with 16-byte loads straight into registers.
template <int KMAX, int ROWS>
__global__ void __launch_bounds__(256) cgemm_rows_regk_kernel(const float2* __restrict__ S, const float2* __restrict__ G,
                                                              float2* __restrict__ C, double2* __restrict__ acc, int ns,
                                                              int ng, int K, int batch, long long s_stride,
                                                              long long g_stride, int tiles_g) {
  // ROWS rows of the large operand per thread (256 * ROWS per CTA): each small-
  // operand value read from shared memory serves ROWS multiply-adds
  __shared__ float2 Ss[RW_SMAX][KMAX];
  const int tile = int(blockIdx.x % tiles_g);
  const int h = int(blockIdx.x / tiles_g);
  const float2* Sh = S + size_t(h) * ns * K;
  for (int i = threadIdx.x; i < RW_SMAX * KMAX; i += blockDim.x) {
    const int r = i / KMAX, kk = i % KMAX;
    Ss[r][kk] = (r < ns && kk < K) ? Sh[size_t(r) * K + kk] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  int g[ROWS];
  bool live[ROWS];
  float2 gv[ROWS][KMAX];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    g[r] = tile * 256 * ROWS + r * 256 + threadIdx.x;
    live[r] = g[r] < ng;
    const float2* row = G + size_t(h) * ng * K + size_t(live[r] ? g[r] : 0) * K;
    if ((K & 1) == 0) {
#pragma unroll
      for (int kk = 0; kk < KMAX; kk += 2)
        if (kk < K) {
          const float4 v = live[r] ? *reinterpret_cast<const float4*>(row + kk) : make_float4(0.f, 0.f, 0.f, 0.f);
          gv[r][kk] = make_float2(v.x, v.y);
          gv[r][kk + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
      for (int kk = 0; kk < KMAX; ++kk)
        if (kk < K) gv[r][kk] = live[r] ? row[kk] : make_float2(0.f, 0.f);
    }
  }
  const size_t hbase = size_t(h) * ns * ng;
#pragma unroll
  for (int s = 0; s < RW_SMAX; ++s) {
    if (s >= ns) break;
    float ar[ROWS], ai[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) ar[r] = ai[r] = 0.f;
#pragma unroll
    for (int kk = 0; kk < KMAX; ++kk) {
      if (kk < K) {
        const float2 a = Ss[s][kk];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          const float2 bb = gv[r][kk];
          ar[r] = fmaf(a.x, bb.x, ar[r]);
          ar[r] = fmaf(-a.y, bb.y, ar[r]);
          ai[r] = fmaf(a.x, bb.y, ai[r]);
          ai[r] = fmaf(a.y, bb.x, ai[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      if (!live[r]) continue;
      const size_t o = hbase + size_t(s) * s_stride + size_t(g[r]) * g_stride;
      if (acc) {
        double2 v = acc[o];
        v.x += ar[r];
        v.y += ai[r];
        acc[o] = v;
      } else {
        C[o] = make_float2(ar[r], ai[r]);
      }
    }
  }
}

// As cgemm_rows_regk_kernel, but the large operand is read in its stored bit
// layout (no separate permute): row g (its N or M index, then batch bits) starts
// at the source offset sum_j bit_j(g) << rowpos[j], and element k of a row is
// koff[k] further on.  Leaves with sliced labels add the slice offset.  The row
// offset is split into the thread's low 8 row bits (computed once) and the
// CTA's row-block bits above them (one deposit per block, in shared memory);
// EXACT instances have K == KMAX at compile time, and the small operand is read
// in 16-byte pairs of k.
template <int KMAX, int ROWS, bool EXACT>
__global__ void __launch_bounds__(256) cgemm_rows_gather_kernel(const float2* __restrict__ S,
                                                                const float2* __restrict__ G, const GatherDesc gd,
                                                                float2* __restrict__ C, double2* __restrict__ acc,
                                                                int ns, int ng, int K, int batch, long long s_stride,
                                                                long long g_stride, int tiles_g, int slice_id) {
  static_assert(KMAX % 2 == 0, "pairs of k");
  __shared__ __align__(16) float2 Ss[RW_SMAX][KMAX];
  __shared__ uint32_t koff[KMAX];
  __shared__ unsigned long long hib[ROWS];
  const int tile = int(blockIdx.x % tiles_g);
  const int h = int(blockIdx.x / tiles_g);
  const float2* Sh = S + size_t(h) * ns * K;
  for (int i = threadIdx.x; i < RW_SMAX * KMAX; i += blockDim.x) {
    const int r = i / KMAX, kk = i % KMAX;
    Ss[r][kk] = (r < ns && kk < K) ? Sh[size_t(r) * K + kk] : make_float2(0.f, 0.f);
  }
  for (int kk = threadIdx.x; kk < KMAX; kk += blockDim.x) {
    uint32_t o = 0;
    for (int j = 0; j < gd.nk; ++j)
      if ((kk >> j) & 1) o |= 1u << gd.kpos[j];
    koff[kk] = o;
  }
  // rows of block r: (tile * ROWS + r) * 256 + threadIdx.x of batch entry h;
  // with ng a multiple of 256 the global row index's low 8 bits are threadIdx.x
  const bool split8 = gd.nrow >= 8 && (ng & 255) == 0;
  if (split8 && threadIdx.x < ROWS) {
    const long long hi = ((long long)h * ng + (long long)(tile * ROWS + int(threadIdx.x)) * 256) >> 8;
    unsigned long long o = 0;
    for (int j = 8; j < gd.nrow; ++j)
      if ((hi >> (j - 8)) & 1) o |= 1ull << gd.rowpos[j];
    hib[threadIdx.x] = o;
  }
  size_t soff = 0;
  for (int j = 0; j < gd.n_slice; ++j)
    if (gd.slice_src[j] >= 0 && ((slice_id >> j) & 1)) soff |= size_t(1) << gd.slice_src[j];
  size_t lo8 = 0;
  if (split8)
    for (int j = 0; j < 8; ++j)
      if ((threadIdx.x >> j) & 1) lo8 |= size_t(1) << gd.rowpos[j];
  __syncthreads();
  const bool pairs = gd.nk >= 1 && gd.kpos[0] == 0;
  int g[ROWS];
  bool live[ROWS];
  float2 gv[ROWS][KMAX];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    g[r] = tile * 256 * ROWS + r * 256 + threadIdx.x;
    live[r] = g[r] < ng;
    size_t base = soff;
    if (split8) {
      base |= lo8 | size_t(hib[r]);
    } else {
      // global row index over (g, h): g's bits first, then the batch bits
      const long long grow = (long long)h * ng + (live[r] ? g[r] : 0);
      for (int j = 0; j < gd.nrow; ++j)
        if ((grow >> j) & 1) base |= size_t(1) << gd.rowpos[j];
    }
    if (pairs) {
      // the lowest K bit is the stored layout's stride-1 bit: pairs (k, k+1) are
      // adjacent and 16-byte aligned (every other offset bit is >= 1)
#pragma unroll
      for (int kk = 0; kk < KMAX; kk += 2) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((EXACT || kk < K) && live[r]) v = *reinterpret_cast<const float4*>(G + base + koff[kk]);
        gv[r][kk] = make_float2(v.x, v.y);
        gv[r][kk + 1] = make_float2(v.z, v.w);
      }
    } else {
#pragma unroll
      for (int kk = 0; kk < KMAX; ++kk)
        gv[r][kk] = ((EXACT || kk < K) && live[r]) ? G[base + koff[kk]] : make_float2(0.f, 0.f);
    }
  }
  size_t obase[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) obase[r] = size_t(h) * ns * ng + size_t(g[r]) * g_stride;
#pragma unroll
  for (int s = 0; s < RW_SMAX; ++s) {
    if (s >= ns) break;
    float ar[ROWS], ai[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) ar[r] = ai[r] = 0.f;
    // values beyond K are zero on both sides, so whole pairs are summed
#pragma unroll
    for (int kk = 0; kk < KMAX; kk += 2) {
      if (EXACT || kk < K) {
        const float4 a2 = *reinterpret_cast<const float4*>(&Ss[s][kk]);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          const float2 b0 = gv[r][kk], b1 = gv[r][kk + 1];
          ar[r] = fmaf(a2.x, b0.x, ar[r]);
          ar[r] = fmaf(-a2.y, b0.y, ar[r]);
          ai[r] = fmaf(a2.x, b0.y, ai[r]);
          ai[r] = fmaf(a2.y, b0.x, ai[r]);
          ar[r] = fmaf(a2.z, b1.x, ar[r]);
          ar[r] = fmaf(-a2.w, b1.y, ar[r]);
          ai[r] = fmaf(a2.z, b1.y, ai[r]);
          ai[r] = fmaf(a2.w, b1.x, ai[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      if (!live[r]) continue;
      const size_t o = obase[r] + size_t(s) * s_stride;
      if (acc) {
        double2 v = acc[o];
        v.x += ar[r];
        v.y += ai[r];
        acc[o] = v;
      } else {
        C[o] = make_float2(ar[r], ai[r]);
      }
    }
  }
}

}  // namespace

cudaError_t launch_cgemm_rows_gather(const void* Ssmall, const void* Gsrc, const GatherDesc& gd, void* C, void* acc,
                                     int ns, int ng, int K, int batch, long long s_stride_out, long long g_stride_out,
                                     int slice_id, cudaStream_t st) {
  if (ns < 1 || ns > RW_SMAX || K > 32 || gd.nrow > 32 || gd.nk > 5) return cudaErrorInvalidConfiguration;
  const int rows = K <= 8 ? 2 : 1;  // rows per thread (more would cut occupancy)
  const long long tg = (ng + 256 * rows - 1) / (256 * rows);
  if (tg * batch > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const dim3 g2{unsigned(tg * batch), 1u, 1u};
  const float2* Sp = reinterpret_cast<const float2*>(Ssmall);
  const float2* Gp = reinterpret_cast<const float2*>(Gsrc);
  float2* Cp = reinterpret_cast<float2*>(C);
  double2* Ap = reinterpret_cast<double2*>(acc);
#define TNQ_GATHER(KM, R, EX)                                                                               \
  cgemm_rows_gather_kernel<KM, R, EX><<<g2, 256, 0, st>>>(Sp, Gp, gd, Cp, Ap, ns, ng, K, batch, s_stride_out,  \
                                                          g_stride_out, int(tg), slice_id)
  switch (K) {
    case 2: TNQ_GATHER(2, 2, true); break;
    case 4: TNQ_GATHER(4, 2, true); break;
    case 8: TNQ_GATHER(8, 2, true); break;
    case 16: TNQ_GATHER(16, 1, true); break;
    case 32: TNQ_GATHER(32, 1, true); break;
    default:
      if (K <= 8) TNQ_GATHER(8, 2, false);
      else if (K <= 16) TNQ_GATHER(16, 1, false);
      else TNQ_GATHER(32, 1, false);
  }
#undef TNQ_GATHER
  return cudaGetLastError();
}

cudaError_t launch_cgemm_rows(const void* Ssmall, const void* Gbig, void* C, void* acc, void* part, int splits,
                              int ns, int ng, int K, int batch, long long s_stride_out, long long g_stride_out,
                              cudaStream_t st) {
  if (ns < 1 || ns > RW_SMAX || splits < 1 || splits > 65535) return cudaErrorInvalidConfiguration;
  if (K <= 32 && splits == 1) {
    // short rows: register-resident rows of the large operand
    const int rows = K <= 8 ? 2 : 1;
    const long long tg = (ng + 256 * rows - 1) / (256 * rows);
    if (tg * batch > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const dim3 g2{unsigned(tg * batch), 1u, 1u};
    const float2* Sp = reinterpret_cast<const float2*>(Ssmall);
    const float2* Gp = reinterpret_cast<const float2*>(Gbig);
    float2* Cp = reinterpret_cast<float2*>(C);
    double2* Ap = reinterpret_cast<double2*>(acc);
    if (K <= 8)
      cgemm_rows_regk_kernel<8, 2><<<g2, 256, 0, st>>>(Sp, Gp, Cp, Ap, ns, ng, K, batch, s_stride_out, g_stride_out, int(tg));
    else if (K <= 16)
      cgemm_rows_regk_kernel<16, 1><<<g2, 256, 0, st>>>(Sp, Gp, Cp, Ap, ns, ng, K, batch, s_stride_out, g_stride_out, int(tg));
    else
      cgemm_rows_regk_kernel<32, 1><<<g2, 256, 0, st>>>(Sp, Gp, Cp, Ap, ns, ng, K, batch, s_stride_out, g_stride_out, int(tg));
    return cudaGetLastError();
  }
  const long long tiles_g = (ng + RW_THREADS - 1) / RW_THREADS;
  if (tiles_g * batch > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  int kchunk = ((K + splits - 1) / splits + RW_KC - 1) / RW_KC * RW_KC;
  dim3 grid{unsigned(tiles_g * batch), unsigned(splits), 1u};
  cgemm_rows_kernel<<<grid, RW_THREADS, 0, st>>>(
      reinterpret_cast<const float2*>(Ssmall), reinterpret_cast<const float2*>(Gbig), reinterpret_cast<float2*>(C),
      reinterpret_cast<double2*>(acc), splits > 1 ? reinterpret_cast<float2*>(part) : nullptr, ns, ng, K, batch,
      s_stride_out, g_stride_out, kchunk, int(tiles_g));
  return cudaGetLastError();
}

DotOp dot_contiguous(const void* p, int rows, int K, int batch) {
  // [batch][rows][K]: K bits lowest, then the row bits, then the batch bits
  DotOp d{};
  d.p = reinterpret_cast<const float2*>(p);
  int nk = 0, nr = 0, nh = 0;
  while ((1 << nk) < K) ++nk;
  while ((1 << nr) < rows) ++nr;
  while ((1 << nh) < batch) ++nh;
  d.nk = nk;
  for (int j = 0; j < nk; ++j) d.kpos[j] = (signed char)j;
  d.nrow = nr + nh;
  for (int j = 0; j < nr + nh; ++j) d.rowpos[j] = (signed char)(nk + j);
  d.kmask = (nk >= 64) ? ~0ull : ((1ull << nk) - 1);
  return d;
}

cudaError_t launch_cdot_ops(const DotOp& A, const DotOp& B, void* part, int splits, int M, int N, int K, int batch,
                            cudaStream_t st) {
  if (M < 1 || M > 8 || N < 1 || N > 8 || splits < 1 || batch > 65535) return cudaErrorInvalidConfiguration;
  // M, N and K are powers of two (all-dim-2 tensors); K bit 0 must be stored
  // bit 0 of both operands for the 16-byte pair loads
  if ((M & (M - 1)) || (N & (N - 1)) || (K & (K - 1)) || K < 2) return cudaErrorInvalidConfiguration;
  if (A.nk < 1 || B.nk < 1 || A.kpos[0] != 0 || B.kpos[0] != 0 || A.nk > 40 || B.nk > 40 || A.nrow > 24 ||
      B.nrow > 24)
    return cudaErrorInvalidConfiguration;
  // K offsets advance by carry-through-mask addition: positions must increase
  for (int j = 1; j < A.nk; ++j)
    if (A.kpos[j] <= A.kpos[j - 1]) return cudaErrorInvalidConfiguration;
  for (int j = 1; j < B.nk; ++j)
    if (B.kpos[j] <= B.kpos[j - 1]) return cudaErrorInvalidConfiguration;
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + 1) & ~1;
  dim3 grid{unsigned(splits), unsigned(batch), 1u};
  float2* Pp = reinterpret_cast<float2*>(part);
  const int tm = M < 4 ? M : 4, tn = N < 4 ? N : 4;
#define TNQ_DOT(TM_, TN_) \
  if (tm == TM_ && tn == TN_) cdot_blk_kernel<TM_, TN_><<<grid, DOT_THREADS, 0, st>>>(A, B, Pp, M, N, K, kchunk)
  TNQ_DOT(1, 1); else TNQ_DOT(1, 2); else TNQ_DOT(1, 4); else TNQ_DOT(2, 1); else TNQ_DOT(2, 2);
  else TNQ_DOT(2, 4); else TNQ_DOT(4, 1); else TNQ_DOT(4, 2); else TNQ_DOT(4, 4);
#undef TNQ_DOT
  return cudaGetLastError();
}

cudaError_t launch_cdot(const void* A, const void* B, void* part, int splits, int M, int N, int K, int batch,
                        cudaStream_t st) {
  return launch_cdot_ops(dot_contiguous(A, M, K, batch), dot_contiguous(B, N, K, batch), part, splits, M, N, K, batch,
                         st);
}

}  // namespace tnq
