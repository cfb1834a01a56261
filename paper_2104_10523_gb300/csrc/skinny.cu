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

// MX x MX complex sums per thread (MX = 4 or 8): register accumulators over the
// thread's part of K, then a fixed-order reduction over the CTA.
template <int MX>
__global__ void __launch_bounds__(DOT_THREADS) cdot_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                                           float2* __restrict__ part, int M, int N, int K,
                                                           int kchunk) {
  __shared__ float red[DOT_THREADS / 32][2 * MX * MX];
  const int split = blockIdx.x, h = blockIdx.y;
  const int kbeg = split * kchunk, kend = min(K, kbeg + kchunk);
  const float2* Ah = A + size_t(h) * M * K;
  const float2* Bh = B + size_t(h) * N * K;
  float cr[MX][MX], ci[MX][MX];
#pragma unroll
  for (int i = 0; i < MX; ++i)
#pragma unroll
    for (int j = 0; j < MX; ++j) cr[i][j] = ci[i][j] = 0.f;
  // two complex values per 16-byte load (kbeg is even because kchunk is)
  for (int k = kbeg + 2 * threadIdx.x; k < kend; k += 2 * DOT_THREADS) {
    const bool two = k + 1 < kend;
    float4 a[MX], b[MX];
#pragma unroll
    for (int i = 0; i < MX; ++i) {
      a[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      b[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < M) {
        if (two) a[i] = *reinterpret_cast<const float4*>(Ah + size_t(i) * K + k);
        else { float2 v = Ah[size_t(i) * K + k]; a[i].x = v.x; a[i].y = v.y; }
      }
      if (i < N) {
        if (two) b[i] = *reinterpret_cast<const float4*>(Bh + size_t(i) * K + k);
        else { float2 v = Bh[size_t(i) * K + k]; b[i].x = v.x; b[i].y = v.y; }
      }
    }
#pragma unroll
    for (int i = 0; i < MX; ++i)
#pragma unroll
      for (int j = 0; j < MX; ++j) {
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
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < MX; ++i)
#pragma unroll
    for (int j = 0; j < MX; ++j) {
      float r = cr[i][j], im = ci[i][j];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        r += __shfl_xor_sync(0xffffffffu, r, off);
        im += __shfl_xor_sync(0xffffffffu, im, off);
      }
      if (lane == 0) {
        red[warp][2 * (i * MX + j)] = r;
        red[warp][2 * (i * MX + j) + 1] = im;
      }
    }
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * MX * MX; q += DOT_THREADS) {
    float v = 0.f;
    for (int w = 0; w < DOT_THREADS / 32; ++w) v += red[w][q];
    const int ij = q >> 1, i = ij / MX, j = ij % MX;
    if (i < M && j < N) {
      float* dst = reinterpret_cast<float*>(part + (size_t(split) * gridDim.y + h) * M * N + size_t(i) * N + j);
      dst[q & 1] = v;
    }
  }
}

// Small operand of ns <= 32 rows and K <= 32: each thread owns one row of the
// large operand and reads it with 16-byte loads straight into registers.
template <int KMAX>
__global__ void __launch_bounds__(256) cgemm_rows_regk_kernel(const float2* __restrict__ S, const float2* __restrict__ G,
                                                              float2* __restrict__ C, double2* __restrict__ acc, int ns,
                                                              int ng, int K, int batch, long long s_stride,
                                                              long long g_stride, int tiles_g) {
  __shared__ float2 Ss[RW_SMAX][KMAX];
  const int tile = int(blockIdx.x % tiles_g);
  const int h = int(blockIdx.x / tiles_g);
  const float2* Sh = S + size_t(h) * ns * K;
  for (int i = threadIdx.x; i < RW_SMAX * KMAX; i += blockDim.x) {
    const int r = i / KMAX, kk = i % KMAX;
    Ss[r][kk] = (r < ns && kk < K) ? Sh[size_t(r) * K + kk] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int g = tile * blockDim.x + threadIdx.x;
  if (g >= ng) return;
  const float2* row = G + size_t(h) * ng * K + size_t(g) * K;
  float2 gv[KMAX];
  if ((K & 1) == 0) {
#pragma unroll
    for (int kk = 0; kk < KMAX; kk += 2)
      if (kk < K) {
        const float4 v = *reinterpret_cast<const float4*>(row + kk);
        gv[kk] = make_float2(v.x, v.y);
        gv[kk + 1] = make_float2(v.z, v.w);
      }
  } else {
#pragma unroll
    for (int kk = 0; kk < KMAX; ++kk)
      if (kk < K) gv[kk] = row[kk];
  }
  const size_t hbase = size_t(h) * ns * ng;
#pragma unroll
  for (int s = 0; s < RW_SMAX; ++s) {
    if (s >= ns) break;
    float ar = 0.f, ai = 0.f;
#pragma unroll
    for (int kk = 0; kk < KMAX; ++kk) {
      if (kk < K) {
        const float2 a = Ss[s][kk], b = gv[kk];
        ar = fmaf(a.x, b.x, ar);
        ar = fmaf(-a.y, b.y, ar);
        ai = fmaf(a.x, b.y, ai);
        ai = fmaf(a.y, b.x, ai);
      }
    }
    const size_t o = hbase + size_t(s) * s_stride + size_t(g) * g_stride;
    if (acc) {
      double2 v = acc[o];
      v.x += ar;
      v.y += ai;
      acc[o] = v;
    } else {
      C[o] = make_float2(ar, ai);
    }
  }
}

// As cgemm_rows_regk_kernel, but the large operand is read in its stored bit
// layout (no separate permute): row g (its N or M index, then batch bits) starts
// at the source offset sum_j bit_j(g) << rowpos[j], and element k of a row is
// koff[k] further on.  Leaves with sliced labels add the slice offset.
template <int KMAX>
__global__ void __launch_bounds__(256) cgemm_rows_gather_kernel(const float2* __restrict__ S,
                                                                const float2* __restrict__ G, const GatherDesc gd,
                                                                float2* __restrict__ C, double2* __restrict__ acc,
                                                                int ns, int ng, int K, int batch, long long s_stride,
                                                                long long g_stride, int tiles_g, int slice_id) {
  __shared__ float2 Ss[RW_SMAX][KMAX];
  __shared__ uint32_t koff[KMAX];
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
  __syncthreads();
  const int g = tile * blockDim.x + threadIdx.x;
  if (g >= ng) return;
  // global row index over (g, h): g's bits first, then the batch bits
  const long long grow = (long long)h * ng + g;
  size_t base = 0;
  for (int j = 0; j < gd.nrow; ++j)
    if ((grow >> j) & 1) base |= size_t(1) << gd.rowpos[j];
  for (int j = 0; j < gd.n_slice; ++j)
    if (gd.slice_src[j] >= 0 && ((slice_id >> j) & 1)) base |= size_t(1) << gd.slice_src[j];
  float2 gv[KMAX];
  if (gd.nk >= 1 && gd.kpos[0] == 0) {
    // the lowest K bit is the stored layout's stride-1 bit: pairs (k, k+1) are
    // adjacent and 16-byte aligned (every other offset bit is >= 1)
#pragma unroll
    for (int kk = 0; kk < KMAX; kk += 2)
      if (kk < K) {
        const float4 v = *reinterpret_cast<const float4*>(G + base + koff[kk]);
        gv[kk] = make_float2(v.x, v.y);
        gv[kk + 1] = make_float2(v.z, v.w);
      }
  } else {
#pragma unroll
    for (int kk = 0; kk < KMAX; ++kk)
      if (kk < K) gv[kk] = G[base + koff[kk]];
  }
  const size_t hbase = size_t(h) * ns * ng;
#pragma unroll
  for (int s = 0; s < RW_SMAX; ++s) {
    if (s >= ns) break;
    float ar = 0.f, ai = 0.f;
#pragma unroll
    for (int kk = 0; kk < KMAX; ++kk) {
      if (kk < K) {
        const float2 a = Ss[s][kk], b = gv[kk];
        ar = fmaf(a.x, b.x, ar);
        ar = fmaf(-a.y, b.y, ar);
        ai = fmaf(a.x, b.y, ai);
        ai = fmaf(a.y, b.x, ai);
      }
    }
    const size_t o = hbase + size_t(s) * s_stride + size_t(g) * g_stride;
    if (acc) {
      double2 v = acc[o];
      v.x += ar;
      v.y += ai;
      acc[o] = v;
    } else {
      C[o] = make_float2(ar, ai);
    }
  }
}

}  // namespace

cudaError_t launch_cgemm_rows_gather(const void* Ssmall, const void* Gsrc, const GatherDesc& gd, void* C, void* acc,
                                     int ns, int ng, int K, int batch, long long s_stride_out, long long g_stride_out,
                                     int slice_id, cudaStream_t st) {
  if (ns < 1 || ns > RW_SMAX || K > 32 || gd.nrow > 32 || gd.nk > 5) return cudaErrorInvalidConfiguration;
  const long long tg = (ng + 255) / 256;
  if (tg * batch > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const dim3 g2{unsigned(tg * batch), 1u, 1u};
  const float2* Sp = reinterpret_cast<const float2*>(Ssmall);
  const float2* Gp = reinterpret_cast<const float2*>(Gsrc);
  float2* Cp = reinterpret_cast<float2*>(C);
  double2* Ap = reinterpret_cast<double2*>(acc);
  if (K <= 8)
    cgemm_rows_gather_kernel<8><<<g2, 256, 0, st>>>(Sp, Gp, gd, Cp, Ap, ns, ng, K, batch, s_stride_out, g_stride_out,
                                                    int(tg), slice_id);
  else if (K <= 16)
    cgemm_rows_gather_kernel<16><<<g2, 256, 0, st>>>(Sp, Gp, gd, Cp, Ap, ns, ng, K, batch, s_stride_out,
                                                     g_stride_out, int(tg), slice_id);
  else
    cgemm_rows_gather_kernel<32><<<g2, 256, 0, st>>>(Sp, Gp, gd, Cp, Ap, ns, ng, K, batch, s_stride_out,
                                                     g_stride_out, int(tg), slice_id);
  return cudaGetLastError();
}

cudaError_t launch_cgemm_rows(const void* Ssmall, const void* Gbig, void* C, void* acc, void* part, int splits,
                              int ns, int ng, int K, int batch, long long s_stride_out, long long g_stride_out,
                              cudaStream_t st) {
  if (ns < 1 || ns > RW_SMAX || splits < 1 || splits > 65535) return cudaErrorInvalidConfiguration;
  if (K <= 32 && splits == 1) {
    // short rows: register-resident row of the large operand
    const long long tg = (ng + 255) / 256;
    if (tg * batch > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const dim3 g2{unsigned(tg * batch), 1u, 1u};
    const float2* Sp = reinterpret_cast<const float2*>(Ssmall);
    const float2* Gp = reinterpret_cast<const float2*>(Gbig);
    float2* Cp = reinterpret_cast<float2*>(C);
    double2* Ap = reinterpret_cast<double2*>(acc);
    if (K <= 8)
      cgemm_rows_regk_kernel<8><<<g2, 256, 0, st>>>(Sp, Gp, Cp, Ap, ns, ng, K, batch, s_stride_out, g_stride_out, int(tg));
    else if (K <= 16)
      cgemm_rows_regk_kernel<16><<<g2, 256, 0, st>>>(Sp, Gp, Cp, Ap, ns, ng, K, batch, s_stride_out, g_stride_out, int(tg));
    else
      cgemm_rows_regk_kernel<32><<<g2, 256, 0, st>>>(Sp, Gp, Cp, Ap, ns, ng, K, batch, s_stride_out, g_stride_out, int(tg));
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

cudaError_t launch_cdot(const void* A, const void* B, void* part, int splits, int M, int N, int K, int batch,
                        cudaStream_t st) {
  if (M < 1 || M > 8 || N < 1 || N > 8 || splits < 1 || batch > 65535) return cudaErrorInvalidConfiguration;
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + 1) & ~1;
  dim3 grid{unsigned(splits), unsigned(batch), 1u};
  const float2* Ap = reinterpret_cast<const float2*>(A);
  const float2* Bp = reinterpret_cast<const float2*>(B);
  float2* Pp = reinterpret_cast<float2*>(part);
  if (M <= 4 && N <= 4)
    cdot_kernel<4><<<grid, DOT_THREADS, 0, st>>>(Ap, Bp, Pp, M, N, K, kchunk);
  else
    cdot_kernel<8><<<grid, DOT_THREADS, 0, st>>>(Ap, Bp, Pp, M, N, K, kchunk);
  return cudaGetLastError();
}

}  // namespace tnq
