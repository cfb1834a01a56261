// Bit-permute, SIMT complex GEMM, projection fill and FP64 finalisation.
//
// Every index has dimension 2, so reordering a tensor's indices is a
// permutation of the bits of its flat element index.  The permute kernel
// stages tiles through shared memory: a tile spans the lowest destination bits
// and the lowest source bits, so both the HBM read and the HBM write run along
// contiguous runs.  It also writes the operand formats the GEMMs want (the real
// expansion of a complex operand, TF32/BF16 hi-lo splits), so a step makes one
// pass over each operand.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.cuh"

namespace tnq {

// ------------------------------------------------------------------ permute
void build_perm_desc(const int* src_labels, int src_rank, const int* dst_labels, int dst_rank,
                     const int* slice_labels, int n_slice, int mode, int kbits, PermDesc* d) {
  std::memset(d, 0, sizeof(*d));
  d->r = dst_rank;
  d->mode = mode;
  d->kbits = kbits;
  d->n_slice = n_slice;
  auto src_pos = [&](int l) {
    for (int p = 0; p < src_rank; ++p)
      if (src_labels[p] == l) return p;
    return -1;
  };
  std::vector<int> s_of_d(dst_rank);
  for (int p = 0; p < dst_rank; ++p) s_of_d[p] = src_pos(dst_labels[p]);
  // a sliced label fixes its source bit to the slice's value, unless the
  // destination keeps it as an index of its own
  auto in_dst = [&](int l) {
    for (int p = 0; p < dst_rank; ++p)
      if (dst_labels[p] == l) return true;
    return false;
  };
  for (int j = 0; j < n_slice; ++j) d->slice_src[j] = in_dst(slice_labels[j]) ? -1 : src_pos(slice_labels[j]);
  for (int j = n_slice; j < 32; ++j) d->slice_src[j] = -1;
  // tile: lowest destination bits and lowest source bits, grown until 11 bits
  int target = std::min(dst_rank, 11);
  std::vector<char> in_tile(dst_rank, 0);
  int u = 0, a = 0, b = 0;
  std::vector<int> d_of_s(src_rank, -1);
  for (int p = 0; p < dst_rank; ++p) d_of_s[s_of_d[p]] = p;
  while (u < target) {
    if (a < dst_rank && (a <= b || b >= src_rank)) {
      if (!in_tile[a]) {
        in_tile[a] = 1;
        ++u;
      }
      ++a;
    } else if (b < src_rank) {
      int p = d_of_s[b];
      if (p >= 0 && !in_tile[p] && u < target) {
        in_tile[p] = 1;
        ++u;
      }
      ++b;
    } else {
      break;
    }
  }
  d->u = u;
  // tile bits in source order
  std::vector<int> tile_dst;  // destination positions of tile bits, in source order
  for (int s = 0; s < src_rank; ++s) {
    int p = d_of_s[s];
    if (p >= 0 && in_tile[p]) tile_dst.push_back(p);
  }
  for (int i = 0; i < u; ++i) d->tile_src[i] = s_of_d[tile_dst[i]];
  std::vector<int> sorted = tile_dst;
  std::sort(sorted.begin(), sorted.end());
  for (int j = 0; j < u; ++j) {
    d->tile_dst_sorted[j] = sorted[j];
    d->tile_srcidx_of_dst[j] =
        int(std::find(tile_dst.begin(), tile_dst.end(), sorted[j]) - tile_dst.begin());
  }
  int k = 0;
  for (int p = 0; p < dst_rank; ++p)
    if (!in_tile[p]) {
      d->outer_dst[k] = p;
      d->outer_src[k] = s_of_d[p];
      ++k;
    }
  d->n_outer = k;
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void write_operand(const PermDesc& d, void* dst0, void* dst1, size_t o,
                                              float2 v) {
  switch (d.mode) {
    case PM_C64:
      reinterpret_cast<float2*>(dst0)[o] = v;
      break;
    case PM_AEXP_F32:
    case PM_AEXP_TF32:
    case PM_AEXP_TF32X3:
    case PM_AEXP_BF16X3: {
      size_t K = size_t(1) << d.kbits;
      size_t row = o >> d.kbits, k = o & (K - 1);
      size_t i0 = (2 * row) * K + k, i1 = (2 * row + 1) * K + k;
      float re = v.x, im = v.y;
      if (d.mode == PM_AEXP_F32) {
        reinterpret_cast<float2*>(dst0)[i0] = make_float2(re, -im);
        reinterpret_cast<float2*>(dst0)[i1] = make_float2(im, re);
      } else if (d.mode == PM_AEXP_TF32) {
        float hr = tf32_round(re), hi = tf32_round(im);
        reinterpret_cast<float2*>(dst0)[i0] = make_float2(hr, -hi);
        reinterpret_cast<float2*>(dst0)[i1] = make_float2(hi, hr);
      } else if (d.mode == PM_AEXP_TF32X3) {
        float hr = tf32_round(re), hi = tf32_round(im);
        float lr = tf32_round(re - hr), li = tf32_round(im - hi);
        reinterpret_cast<float2*>(dst0)[i0] = make_float2(hr, -hi);
        reinterpret_cast<float2*>(dst0)[i1] = make_float2(hi, hr);
        reinterpret_cast<float2*>(dst1)[i0] = make_float2(lr, -li);
        reinterpret_cast<float2*>(dst1)[i1] = make_float2(li, lr);
      } else {
        __nv_bfloat16 hr = __float2bfloat16_rn(re), hi = __float2bfloat16_rn(im);
        __nv_bfloat16 lr = __float2bfloat16_rn(re - __bfloat162float(hr));
        __nv_bfloat16 li = __float2bfloat16_rn(im - __bfloat162float(hi));
        __nv_bfloat162 h0, h1, l0, l1;
        h0.x = hr; h0.y = __hneg(hi);
        h1.x = hi; h1.y = hr;
        l0.x = lr; l0.y = __hneg(li);
        l1.x = li; l1.y = lr;
        reinterpret_cast<__nv_bfloat162*>(dst0)[i0] = h0;
        reinterpret_cast<__nv_bfloat162*>(dst0)[i1] = h1;
        reinterpret_cast<__nv_bfloat162*>(dst1)[i0] = l0;
        reinterpret_cast<__nv_bfloat162*>(dst1)[i1] = l1;
      }
      break;
    }
    case PM_B_TF32:
      reinterpret_cast<float2*>(dst0)[o] = make_float2(tf32_round(v.x), tf32_round(v.y));
      break;
    case PM_B_TF32X3: {
      float hr = tf32_round(v.x), hi = tf32_round(v.y);
      reinterpret_cast<float2*>(dst0)[o] = make_float2(hr, hi);
      reinterpret_cast<float2*>(dst1)[o] = make_float2(tf32_round(v.x - hr), tf32_round(v.y - hi));
      break;
    }
    case PM_B_BF16X3: {
      __nv_bfloat162 h, l;
      h.x = __float2bfloat16_rn(v.x);
      h.y = __float2bfloat16_rn(v.y);
      l.x = __float2bfloat16_rn(v.x - __bfloat162float(h.x));
      l.y = __float2bfloat16_rn(v.y - __bfloat162float(h.y));
      reinterpret_cast<__nv_bfloat162*>(dst0)[o] = h;
      reinterpret_cast<__nv_bfloat162*>(dst1)[o] = l;
      break;
    }
  }
}

constexpr int PERM_THREADS = 256;

__global__ void __launch_bounds__(PERM_THREADS) permute_kernel(const PermDesc d, const float2* __restrict__ src,
                                                               void* dst0, void* dst1, int slice_id) {
  __shared__ float2 tile[2048];
  __shared__ uint32_t srcoff[2048];
  __shared__ uint32_t dstoff[2048];
  __shared__ uint16_t eidx[2048];
  const int T = 1 << d.u;
  for (int e = threadIdx.x; e < T; e += blockDim.x) {
    uint32_t s = 0, o = 0, ei = 0;
    for (int i = 0; i < d.u; ++i)
      if ((e >> i) & 1) {
        s |= 1u << d.tile_src[i];
        o |= 1u << d.tile_dst_sorted[i];
        ei |= 1u << d.tile_srcidx_of_dst[i];
      }
    srcoff[e] = s;
    dstoff[e] = o;
    eidx[e] = (uint16_t)ei;
  }
  size_t slice_off = 0;
  for (int j = 0; j < d.n_slice; ++j)
    if (d.slice_src[j] >= 0 && ((slice_id >> j) & 1)) slice_off |= size_t(1) << d.slice_src[j];
  __syncthreads();
  const size_t n_outer = size_t(1) << d.n_outer;
  for (size_t c = blockIdx.x; c < n_outer; c += gridDim.x) {
    size_t sb = slice_off, db = 0;
    for (int k = 0; k < d.n_outer; ++k)
      if ((c >> k) & 1) {
        sb |= size_t(1) << d.outer_src[k];
        db |= size_t(1) << d.outer_dst[k];
      }
    for (int e = threadIdx.x; e < T; e += blockDim.x) tile[e] = src[sb + srcoff[e]];
    __syncthreads();
    for (int f = threadIdx.x; f < T; f += blockDim.x) write_operand(d, dst0, dst1, db + dstoff[f], tile[eidx[f]]);
    __syncthreads();
  }
}

// Vectorised variant: pairs of elements adjacent in the source (tile bit 0 is
// source bit 0) are loaded with one 16-byte load, pairs adjacent in the
// destination (tile bit 0 in destination order is destination bit 0) are
// stored with one 16-byte store (8 bytes for BF16 formats).  The shared tile is
// XOR-swizzled on bits 1-3 by higher bits so the transposed reads of a
// half-warp spread over the banks while pairs stay adjacent.
__device__ __forceinline__ uint32_t swz(uint32_t e) { return e ^ ((((e >> 4) ^ (e >> 8)) & 7u) << 1); }

__device__ __forceinline__ void write_pair(const PermDesc& d, void* dst0, void* dst1, size_t o, float2 v0, float2 v1) {
  switch (d.mode) {
    case PM_C64:
      *reinterpret_cast<float4*>(reinterpret_cast<float2*>(dst0) + o) = make_float4(v0.x, v0.y, v1.x, v1.y);
      break;
    case PM_B_TF32: {
      *reinterpret_cast<float4*>(reinterpret_cast<float2*>(dst0) + o) =
          make_float4(tf32_round(v0.x), tf32_round(v0.y), tf32_round(v1.x), tf32_round(v1.y));
      break;
    }
    case PM_B_TF32X3: {
      const float h0 = tf32_round(v0.x), h1 = tf32_round(v0.y), h2 = tf32_round(v1.x), h3 = tf32_round(v1.y);
      *reinterpret_cast<float4*>(reinterpret_cast<float2*>(dst0) + o) = make_float4(h0, h1, h2, h3);
      *reinterpret_cast<float4*>(reinterpret_cast<float2*>(dst1) + o) =
          make_float4(tf32_round(v0.x - h0), tf32_round(v0.y - h1), tf32_round(v1.x - h2), tf32_round(v1.y - h3));
      break;
    }
    case PM_B_BF16X3: {
      __nv_bfloat162 a, b, la, lb;
      a.x = __float2bfloat16_rn(v0.x);
      a.y = __float2bfloat16_rn(v0.y);
      b.x = __float2bfloat16_rn(v1.x);
      b.y = __float2bfloat16_rn(v1.y);
      la.x = __float2bfloat16_rn(v0.x - __bfloat162float(a.x));
      la.y = __float2bfloat16_rn(v0.y - __bfloat162float(a.y));
      lb.x = __float2bfloat16_rn(v1.x - __bfloat162float(b.x));
      lb.y = __float2bfloat16_rn(v1.y - __bfloat162float(b.y));
      uint2 hv, lv;
      hv.x = *reinterpret_cast<uint32_t*>(&a);
      hv.y = *reinterpret_cast<uint32_t*>(&b);
      lv.x = *reinterpret_cast<uint32_t*>(&la);
      lv.y = *reinterpret_cast<uint32_t*>(&lb);
      *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat162*>(dst0) + o) = hv;
      *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat162*>(dst1) + o) = lv;
      break;
    }
    default: {  // A' expansion: o and o+1 are consecutive k of the same complex row
      const size_t K = size_t(1) << d.kbits;
      const size_t row = o >> d.kbits, k = o & (K - 1);
      const size_t i0 = (2 * row) * K + k, i1 = (2 * row + 1) * K + k;
      if (d.mode == PM_AEXP_F32 || d.mode == PM_AEXP_TF32) {
        float r0 = v0.x, m0 = v0.y, r1 = v1.x, m1 = v1.y;
        if (d.mode == PM_AEXP_TF32) {
          r0 = tf32_round(r0);
          m0 = tf32_round(m0);
          r1 = tf32_round(r1);
          m1 = tf32_round(m1);
        }
        *reinterpret_cast<float4*>(reinterpret_cast<float2*>(dst0) + i0) = make_float4(r0, -m0, r1, -m1);
        *reinterpret_cast<float4*>(reinterpret_cast<float2*>(dst0) + i1) = make_float4(m0, r0, m1, r1);
      } else if (d.mode == PM_AEXP_TF32X3) {
        const float r0 = tf32_round(v0.x), m0 = tf32_round(v0.y), r1 = tf32_round(v1.x), m1 = tf32_round(v1.y);
        const float lr0 = tf32_round(v0.x - r0), lm0 = tf32_round(v0.y - m0), lr1 = tf32_round(v1.x - r1),
                    lm1 = tf32_round(v1.y - m1);
        *reinterpret_cast<float4*>(reinterpret_cast<float2*>(dst0) + i0) = make_float4(r0, -m0, r1, -m1);
        *reinterpret_cast<float4*>(reinterpret_cast<float2*>(dst0) + i1) = make_float4(m0, r0, m1, r1);
        *reinterpret_cast<float4*>(reinterpret_cast<float2*>(dst1) + i0) = make_float4(lr0, -lm0, lr1, -lm1);
        *reinterpret_cast<float4*>(reinterpret_cast<float2*>(dst1) + i1) = make_float4(lm0, lr0, lm1, lr1);
      } else {  // PM_AEXP_BF16X3
        __nv_bfloat16 r0 = __float2bfloat16_rn(v0.x), m0 = __float2bfloat16_rn(v0.y);
        __nv_bfloat16 r1 = __float2bfloat16_rn(v1.x), m1 = __float2bfloat16_rn(v1.y);
        __nv_bfloat16 lr0 = __float2bfloat16_rn(v0.x - __bfloat162float(r0));
        __nv_bfloat16 lm0 = __float2bfloat16_rn(v0.y - __bfloat162float(m0));
        __nv_bfloat16 lr1 = __float2bfloat16_rn(v1.x - __bfloat162float(r1));
        __nv_bfloat16 lm1 = __float2bfloat16_rn(v1.y - __bfloat162float(m1));
        __nv_bfloat162 p00, p01, p10, p11, q00, q01, q10, q11;
        p00.x = r0; p00.y = __hneg(m0); p01.x = r1; p01.y = __hneg(m1);     // row (m, re), hi
        p10.x = m0; p10.y = r0; p11.x = m1; p11.y = r1;                     // row (m, im), hi
        q00.x = lr0; q00.y = __hneg(lm0); q01.x = lr1; q01.y = __hneg(lm1); // lo parts
        q10.x = lm0; q10.y = lr0; q11.x = lm1; q11.y = lr1;
        uint2 w;
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(dst0);
        __nv_bfloat162* l = reinterpret_cast<__nv_bfloat162*>(dst1);
        w.x = *reinterpret_cast<uint32_t*>(&p00); w.y = *reinterpret_cast<uint32_t*>(&p01);
        *reinterpret_cast<uint2*>(h + i0) = w;
        w.x = *reinterpret_cast<uint32_t*>(&p10); w.y = *reinterpret_cast<uint32_t*>(&p11);
        *reinterpret_cast<uint2*>(h + i1) = w;
        w.x = *reinterpret_cast<uint32_t*>(&q00); w.y = *reinterpret_cast<uint32_t*>(&q01);
        *reinterpret_cast<uint2*>(l + i0) = w;
        w.x = *reinterpret_cast<uint32_t*>(&q10); w.y = *reinterpret_cast<uint32_t*>(&q11);
        *reinterpret_cast<uint2*>(l + i1) = w;
      }
    }
  }
}

constexpr int PV_THREADS = 256;

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst))),
               "l"(gsrc)
               : "memory");
}

// Tiles are double-buffered: the 16-byte loads of the CTA's next tile land in
// shared memory (cp.async) while the current tile is written out.
__global__ void __launch_bounds__(PV_THREADS) permute_vec_kernel(const PermDesc d, const float2* __restrict__ src,
                                                                 void* dst0, void* dst1, int slice_id) {
  __shared__ __align__(16) float2 tile[2][2048];
  __shared__ uint32_t srcoff[1024];   // per source-order pair
  __shared__ uint32_t dstoff[1024];   // per destination-order pair
  __shared__ uint16_t epos[2048];     // per destination-order element: swizzled tile position
  const int T = 1 << d.u, P = T >> 1;
  for (int q = threadIdx.x; q < P; q += blockDim.x) {
    const int e = q << 1;  // even element in source order
    uint32_t s = 0, o = 0;
    for (int i = 1; i < d.u; ++i)
      if ((e >> i) & 1) {
        s |= 1u << d.tile_src[i];
        o |= 1u << d.tile_dst_sorted[i];
      }
    srcoff[q] = s;
    dstoff[q] = o;  // destination offset of the even element of pair q in destination order
  }
  for (int f = threadIdx.x; f < T; f += blockDim.x) {
    uint32_t ei = 0;
    for (int i = 0; i < d.u; ++i)
      if ((f >> i) & 1) ei |= 1u << d.tile_srcidx_of_dst[i];
    epos[f] = (uint16_t)swz(ei);
  }
  size_t slice_off = 0;
  for (int j = 0; j < d.n_slice; ++j)
    if (d.slice_src[j] >= 0 && ((slice_id >> j) & 1)) slice_off |= size_t(1) << d.slice_src[j];
  __syncthreads();
  const size_t n_outer = size_t(1) << d.n_outer;
  auto outer = [&](size_t c, const int* pos) {
    size_t o = 0;
    for (int k = 0; k < d.n_outer; ++k)
      if ((c >> k) & 1) o |= size_t(1) << pos[k];
    return o;
  };
  auto issue = [&](size_t c, int b) {
    const size_t sb = slice_off | outer(c, d.outer_src);
    for (int q = threadIdx.x; q < P; q += blockDim.x) cp_async16(&tile[b][swz(uint32_t(q) << 1)], src + sb + srcoff[q]);
  };
  int b = 0;
  if (size_t(blockIdx.x) < n_outer) issue(blockIdx.x, 0);
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (size_t c = blockIdx.x; c < n_outer; c += gridDim.x) {
    const size_t cn = c + gridDim.x;
    if (cn < n_outer) issue(cn, b ^ 1);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // tile c has landed (this thread's part)
    __syncthreads();
    const size_t db = outer(c, d.outer_dst);
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
      const int f = q << 1;
      write_pair(d, dst0, dst1, db + dstoff[q], tile[b][epos[f]], tile[b][epos[f + 1]]);
    }
    __syncthreads();  // buffer b is refilled by the next iteration's issue
    b ^= 1;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

bool perm_vec_ok(const PermDesc& d) {
  // pairs: source bit 0 and destination bit 0 are both the tile's first bit,
  // and A' expansions keep a pair inside one row (at least two K elements)
  if (d.u < 2 || d.tile_src[0] != 0 || d.tile_dst_sorted[0] != 0) return false;
  if (d.mode >= PM_AEXP_F32 && d.mode <= PM_AEXP_BF16X3 && d.kbits < 1) return false;
  return true;
}

cudaError_t launch_permute(const PermDesc& d, const void* src, void* dst0, void* dst1, int slice_id,
                           int sm_count, cudaStream_t st) {
  size_t n_outer = size_t(1) << d.n_outer;
  if (perm_vec_ok(d)) {
    // persistent CTAs: as many as are resident at once
    static int per_sm = 0;
    if (per_sm == 0) {
      int n = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, permute_vec_kernel, PV_THREADS, 0) != cudaSuccess || n < 1)
        n = 4;
      per_sm = n;
    }
    size_t grid = std::min<size_t>(n_outer, size_t(sm_count) * per_sm);
    permute_vec_kernel<<<(unsigned)grid, PV_THREADS, 0, st>>>(d, reinterpret_cast<const float2*>(src), dst0, dst1,
                                                             slice_id);
    return cudaGetLastError();
  }
  size_t grid = std::min<size_t>(n_outer, size_t(sm_count) * 8);
  permute_kernel<<<(unsigned)grid, PERM_THREADS, 0, st>>>(d, reinterpret_cast<const float2*>(src), dst0,
                                                          dst1, slice_id);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ SIMT complex GEMM
// 64x64 complex tile per CTA, 16-deep K slices in shared memory, 4x4 complex
// outputs per thread (strided so that shared-memory reads and global stores are
// conflict-free and coalesced).
constexpr int SG_BM = 64, SG_BN = 64, SG_BK = 16;

__global__ void __launch_bounds__(256) cgemm_simt_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                                         float2* __restrict__ C, double2* __restrict__ acc,
                                                         float2* __restrict__ part, int M, int N, int K, int batch,
                                                         int kchunk) {
  __shared__ float2 As[SG_BK][SG_BM + 1];
  __shared__ float2 Bs[SG_BK][SG_BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int tiles_n = (N + SG_BN - 1) / SG_BN;
  const int n0 = int(blockIdx.x % tiles_n) * SG_BN, m0 = int(blockIdx.x / tiles_n) * SG_BM;
  for (int h = blockIdx.z; h < batch; h += gridDim.z) {
    const float2* Ah = A + size_t(h) * M * K;
    const float2* Bh = B + size_t(h) * N * K;
    float cr[4][4], ci[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) cr[i][j] = ci[i][j] = 0.f;
    const int kbeg = blockIdx.y * kchunk, kend = min(K, kbeg + kchunk);
    for (int k0 = kbeg; k0 < kend; k0 += SG_BK) {
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        int idx = tid + 256 * l, r = idx >> 4, kk = idx & 15;
        float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
        if (m0 + r < M && k0 + kk < kend) va = Ah[size_t(m0 + r) * K + k0 + kk];
        if (n0 + r < N && k0 + kk < kend) vb = Bh[size_t(n0 + r) * K + k0 + kk];
        As[kk][r] = va;
        Bs[kk][r] = vb;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < SG_BK; ++kk) {
        float2 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            cr[i][j] = fmaf(a[i].x, b[j].x, cr[i][j]);
            cr[i][j] = fmaf(-a[i].y, b[j].y, cr[i][j]);
            ci[i][j] = fmaf(a[i].x, b[j].y, ci[i][j]);
            ci[i][j] = fmaf(a[i].y, b[j].x, ci[i][j]);
          }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
        if (m < M && n < N) {
          size_t o = size_t(h) * M * N + size_t(m) * N + n;
          if (part) {
            part[size_t(blockIdx.y) * batch * M * N + o] = make_float2(cr[i][j], ci[i][j]);
          } else if (acc) {
            double2 t = acc[o];
            t.x += (double)cr[i][j];
            t.y += (double)ci[i][j];
            acc[o] = t;
          } else {
            C[o] = make_float2(cr[i][j], ci[i][j]);
          }
        }
      }
  }
}

cudaError_t launch_cgemm_simt(const void* A, const void* B, void* C, void* acc, void* part, int splits, int M,
                              int N, int K, int batch, cudaStream_t st) {
  size_t tiles = size_t((N + SG_BN - 1) / SG_BN) * size_t((M + SG_BM - 1) / SG_BM);
  if (tiles > 0x7fffffffu || splits < 1 || splits > 65535) return cudaErrorInvalidConfiguration;
  // each split covers a whole number of 16-deep K slices
  int kchunk = ((K + splits - 1) / splits + SG_BK - 1) / SG_BK * SG_BK;
  dim3 grid((unsigned)tiles, (unsigned)splits, std::min(batch, 65535));
  cgemm_simt_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const float2*>(A), reinterpret_cast<const float2*>(B),
                                          reinterpret_cast<float2*>(C), reinterpret_cast<double2*>(acc),
                                          splits > 1 ? reinterpret_cast<float2*>(part) : nullptr, M, N, K, batch,
                                          kchunk);
  return cudaGetLastError();
}

// out = sum over s of part[s] in ascending s (FP32), or acc += that sum in FP64.
__global__ void reduce_splits_kernel(const float2* __restrict__ part, int splits, size_t n, float2* __restrict__ C,
                                     double2* __restrict__ acc) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    if (acc) {
      double re = 0, im = 0;
      for (int s = 0; s < splits; ++s) {
        float2 v = part[size_t(s) * n + i];
        re += v.x;
        im += v.y;
      }
      double2 t = acc[i];
      t.x += re;
      t.y += im;
      acc[i] = t;
    } else {
      float re = 0.f, im = 0.f;
      for (int s = 0; s < splits; ++s) {
        float2 v = part[size_t(s) * n + i];
        re += v.x;
        im += v.y;
      }
      C[i] = make_float2(re, im);
    }
  }
}

cudaError_t launch_reduce_splits(const void* part, int splits, size_t n, void* C, void* acc, int sm_count,
                                 cudaStream_t st) {
  size_t blocks = std::min<size_t>((n + 255) / 256, size_t(sm_count) * 8);
  if (blocks < 1) blocks = 1;
  reduce_splits_kernel<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<const float2*>(part), splits, n,
                                                         reinterpret_cast<float2*>(C), reinterpret_cast<double2*>(acc));
  return cudaGetLastError();
}

// ------------------------------------------------------------------ projection fill
// Projection leaf j (at base + j * stride) gets P[x, b] = [bits[b][src[j]] == x]
// (Sec. 3.1.1: <x_q| closes the qubit's final wire; b enumerates the bitstrings
// of the pass).  Entries tab[n_proj .. n_proj + n_open) name the row entries of
// open qubits, which must hold -1.  Any other value sets *err.
__global__ void proj_fill_kernel(char* base, size_t stride, int n_proj, int n_open, const int* __restrict__ tab,
                                 int row_len, int w, const int8_t* __restrict__ bits, int64_t n_valid, int* err) {
  const int64_t per = int64_t(1) << w;
  const int64_t total = per * (n_proj + n_open);
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int j = int(t / per);
    const int64_t b = t % per;
    const int src = tab[j];
    if (j >= n_proj) {
      if (b < n_valid && bits[b * row_len + src] != -1) atomicOr(err, 1);
      continue;
    }
    float2* P = reinterpret_cast<float2*>(base + stride * j);
    float v0 = 0.f, v1 = 0.f;
    if (b < n_valid) {
      int8_t x = bits[b * row_len + src];
      if (x == 0) v0 = 1.f;
      else if (x == 1) v1 = 1.f;
      else atomicOr(err, 1);
    }
    P[2 * b] = make_float2(v0, 0.f);
    P[2 * b + 1] = make_float2(v1, 0.f);
  }
}

cudaError_t launch_proj_fill(void* leaves_base, size_t stride_bytes, int n_proj, int n_open, const int* tab,
                             int row_len, int batch_log2, const int8_t* bits, int64_t n_valid, int* err_flag,
                             cudaStream_t st) {
  int64_t total = (int64_t(1) << batch_log2) * (n_proj + n_open);
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  if (blocks < 1) return cudaSuccess;
  proj_fill_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<char*>(leaves_base), stride_bytes, n_proj, n_open, tab,
                                           row_len, batch_log2, bits, n_valid, err_flag);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ finalize
struct PosTable {
  int n, n_open;
  int pos[32];
  int open_pos[32];
};

// out[b * 2^n_open + o] = acc[root index of (b, o)]: bit j of b sits at root
// position pos[j]; open qubit i (i = 0 most significant in o) at open_pos[i].
__global__ void finalize_kernel(const double2* __restrict__ acc, void* __restrict__ out, int64_t n_valid, PosTable pt,
                                int real_only) {
  const int64_t total = n_valid << pt.n_open;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = e >> pt.n_open;
    const int64_t o = e & ((int64_t(1) << pt.n_open) - 1);
    size_t r = 0;
    for (int j = 0; j < pt.n; ++j)
      if ((b >> j) & 1) r |= size_t(1) << pt.pos[j];
    for (int i = 0; i < pt.n_open; ++i)
      if ((o >> (pt.n_open - 1 - i)) & 1) r |= size_t(1) << pt.open_pos[i];
    if (real_only)
      reinterpret_cast<double*>(out)[e] = acc[r].x;
    else
      reinterpret_cast<double2*>(out)[e] = acc[r];
  }
}

cudaError_t launch_finalize(const void* acc, void* out, int64_t n_valid, const int* pos_table, int n_pos,
                            const int* open_pos, int n_open, bool real_only, cudaStream_t st) {
  PosTable pt;
  pt.n = n_pos;
  pt.n_open = n_open;
  for (int j = 0; j < n_pos && j < 32; ++j) pt.pos[j] = pos_table[j];
  for (int j = 0; j < n_open && j < 32; ++j) pt.open_pos[j] = open_pos[j];
  const int64_t total = n_valid << n_open;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  if (blocks < 1) blocks = 1;
  finalize_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const double2*>(acc), out, n_valid, pt, real_only ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st) { return cudaMemsetAsync(p, 0, bytes, st); }

}  // namespace tnq
