// Complex GEMM on the 5th-generation tensor cores (tcgen05 + TMEM), sm_103a.
//
// A step of the contraction sequence (Sec. 3.1) is C[h][m][n] =
// sum_k A[h][m][k] B[h][n][k] in complex arithmetic.  It runs as one real GEMM
// D = A' * B^T with
//   A' (2M x 2K):  row (m, re) = [ar_0, -ai_0, ar_1, -ai_1, ...]
//                  row (m, im) = [ai_0,  ar_0, ai_1,  ar_1, ...]
//   B  (N  x 2K):  row n = [br_0, bi_0, br_1, bi_1, ...]  (complex64 as stored)
// so D[(m, re)][n] = Re C[m][n] and D[(m, im)][n] = Im C[m][n]: 8MNK real flops,
// the same count as four real GEMMs, in one K-major contraction.
//
// Precision modes (TF32 is the paper's A100 tensor-core mode, Table 2):
//   TF32    one kind::tf32 product;
//   TF32x3  x = hi + lo with hi, lo TF32: A_lo B_hi + A_hi B_lo + A_hi B_hi;
//   BF16x3  the same split with BF16 parts and kind::f16 (bf16 inputs).
// The tensor-memory accumulator adds each MMA's result with truncation, so its
// error grows linearly with the number of MMAs.  The split modes therefore
// accumulate only `chunk_kb` K blocks at a time in TMEM (two buffers, so the
// MMAs run on while one is drained) and the epilogue warps add each chunk into
// FP32 registers with round-to-nearest; the error then grows with the square
// root of the number of chunks.
//
// CTA = 10 warps: warp 0 issues TMA loads into a ring of shared-memory stages,
// warp 1 allocates TMEM and (one thread) issues the MMAs, warps 2-9 read the
// 128 x BN accumulator back with tcgen05.ld (warp w reads TMEM lanes
// 32*(w%4)..+31, warps 2-5 the left half of the columns, 6-9 the right half)
// and write complex64 (or add FP64 into the cross-slice accumulator).  Every mbarrier wait is bounded; a wait
// that runs out sets the error flag and the CTA unwinds.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "gemm_tc.cuh"
#include "tc_ptx.cuh"
#include "../../include/tnq.h"

namespace tnq {

namespace {

using namespace tcx;

constexpr int TC_THREADS = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int TC_BM = 128;            // rows of A' per tile (64 complex rows)
constexpr int TC_ROW_BYTES = 128;     // one 128B swizzle atom of K per stage
constexpr int TC_MAX_STAGES = 8;
constexpr int TC_SMEM_BUDGET = 200 * 1024;
constexpr int TC_GROUP_M = 16;         // m-tiles per launch-order group

struct TcParams {
  int M;          // complex rows per batch (A' has 2M rows)
  int N;          // rows of B per batch
  int nkb;        // K blocks of 128 bytes
  int tiles_m, tiles_n;
  int BN;
  int split;      // 0: one product; 1: three products (hi/lo)
  int kind_bf16;  // 0: kind::tf32; 1: kind::f16 with bf16 inputs
  int stages;
  int chunk_kb;   // K blocks per TMEM accumulation chunk (>= nkb: one chunk)
  int splits;     // K ranges computed by separate CTAs (1: no split)
  int kb_per_split;
  float2* part;   // splits > 1: FP32 partial products [split][batch][M][N]
  int batch;
  uint32_t idesc;
  uint32_t stage_tx;  // bytes landed per stage
  uint32_t a_bytes, b_bytes;
  float2* C;
  double2* acc;
  int* err;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    cgemm_tc_kernel(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
                    const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
                    const TcParams P) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[TC_MAX_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[TC_MAX_STAGES];
  __shared__ __align__(8) uint64_t acc_full[2];
  __shared__ __align__(8) uint64_t acc_empty[2];
  __shared__ __align__(8) uint64_t final_bar;
  __shared__ uint32_t tmem_slot;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long tiles = (long long)P.tiles_m * P.tiles_n;
  const long long total_tiles = tiles * P.splits * P.batch;
  const uint32_t stage_bytes = (P.split ? 2u : 1u) * (P.a_bytes + P.b_bytes);
  const uint32_t buf_cols = uint32_t(P.BN);
  const uint32_t tmem_cols = 2 * buf_cols < 32 ? 32u : 2 * buf_cols;  // two accumulator buffers

  // Tile t -> (m-tile, n-tile, split, batch).  Within each (split, batch) the
  // output tiles go in groups of TC_GROUP_M m-tiles with the n-tiles swept
  // inside a group, so the CTAs of one wave share A' tile rows and B tiles in L2.
  auto decode = [&](long long t, int* mt, int* nt, int* split, int* h, int* kb0, int* nkb) {
    const int pid = int(t % tiles);
    long long r = t / tiles;
    *split = int(r % P.splits);
    *h = int(r / P.splits);
    const int per_group = TC_GROUP_M * P.tiles_n;
    const int first_m = (pid / per_group) * TC_GROUP_M;
    const int group_m = min(P.tiles_m - first_m, TC_GROUP_M);
    *mt = first_m + (pid % per_group) % group_m;
    *nt = (pid % per_group) / group_m;
    *kb0 = *split * P.kb_per_split;
    *nkb = min(P.nkb - *kb0, P.kb_per_split);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), 8);  // one arrival per epilogue warp
    }
    mbar_init(smem_u32(&final_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: one ring of stages across all tiles of this CTA
    const int k_elems = P.kind_bf16 ? 64 : 32;
    int s = 0;          // ring position and its phase, advanced per K block
    uint32_t ph = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
      int mt, nt, split, h, kb0, nkb;
      decode(t, &mt, &nt, &split, &h, &kb0, &nkb);
      for (int kb = 0; kb < nkb; ++kb) {
        if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1)) {
          atomicOr(P.err, 1);
          ok = false;
          break;
        }
        uint8_t* st = smem + size_t(s) * stage_bytes;
        const uint32_t fb = smem_u32(&full_bar[s]);
        mbar_expect_tx(fb, stage_bytes);
        const int kc = (kb0 + kb) * k_elems;
        tma_load_3d(smem_u32(st), &ta_hi, kc, mt * TC_BM, h, fb);
        tma_load_3d(smem_u32(st + P.a_bytes), &tb_hi, kc, nt * P.BN, h, fb);
        if (P.split) {
          uint8_t* a_lo = st + P.a_bytes + P.b_bytes;
          tma_load_3d(smem_u32(a_lo), &ta_lo, kc, mt * TC_BM, h, fb);
          tma_load_3d(smem_u32(a_lo + P.a_bytes), &tb_lo, kc, nt * P.BN, h, fb);
        }
        if (++s == P.stages) {
          s = 0;
          ph ^= 1;
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: accumulation chunks alternate between the two
    // TMEM buffers across chunk and tile boundaries
    int s = 0, b = 0;           // ring position / accumulator buffer
    uint32_t ph = 0;            // ring phase
    int uses[2] = {0, 0};       // chunks issued so far on each accumulator buffer
    int chunk = 0, kc = 0;      // chunks issued; K blocks into the current chunk
    bool ok = true;
    for (long long t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
      int mt, nt, split, h, kb0, nkb;
      decode(t, &mt, &nt, &split, &h, &kb0, &nkb);
      kc = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const bool chunk_start = kc == 0;
        if (chunk_start) {
          b = chunk & 1;
          // use u >= 1 of buffer b waits for the epilogue's drain of use u - 1,
          // the (u-1)-th completion of acc_empty[b]
          if (uses[b] >= 1 && !mbar_wait(smem_u32(&acc_empty[b]), uint32_t(uses[b] - 1) & 1)) {
            atomicOr(P.err, 1);
            ok = false;
            break;
          }
        }
        if (!mbar_wait(smem_u32(&full_bar[s]), ph)) {
          atomicOr(P.err, 1);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint8_t* st = smem + size_t(s) * stage_bytes;
        const uint32_t a_hi = smem_u32(st), b_hi = smem_u32(st + P.a_bytes);
        const uint32_t a_lo = smem_u32(st + P.a_bytes + P.b_bytes), b_lo = a_lo + P.a_bytes;
        const uint32_t d = tmem + uint32_t(b) * buf_cols;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t off = kk * 32;
          const uint32_t first = (chunk_start && kk == 0) ? 0u : 1u;
          if (P.split) {
            mma_issue(P.kind_bf16, d, smem_desc(a_lo + off), smem_desc(b_hi + off), P.idesc, first);
            mma_issue(P.kind_bf16, d, smem_desc(a_hi + off), smem_desc(b_lo + off), P.idesc, 1u);
            mma_issue(P.kind_bf16, d, smem_desc(a_hi + off), smem_desc(b_hi + off), P.idesc, 1u);
          } else {
            mma_issue(P.kind_bf16, d, smem_desc(a_hi + off), smem_desc(b_hi + off), P.idesc, first);
          }
        }
        mma_commit(smem_u32(&empty_bar[s]));
        if (++s == P.stages) {
          s = 0;
          ph ^= 1;
        }
        if (++kc == P.chunk_kb || kb == nkb - 1) {
          mma_commit(smem_u32(&acc_full[b]));
          ++uses[b];
          ++chunk;
          kc = 0;
        }
      }
    }
    mma_commit(smem_u32(&final_bar));
  } else if (warp >= 2) {
    // ---------------- epilogue: drain every chunk into FP32 registers (round to
    // nearest), write each finished tile
    const int quarter = warp & 3;        // TMEM lanes 32*quarter .. +31 belong to this warp
    const int half = (warp - 2) >> 2;    // which half of the BN columns
    const int nq_all = P.BN / 32;        // 32-column groups in the tile
    const int nq_half = (nq_all + 1) / 2;
    const int q0 = half * nq_half;
    const int nq = min(nq_all - q0, nq_half);  // groups owned by this warp (0..4)
    const uint32_t lane_addr = uint32_t(quarter * 32) << 16;
    const int row = quarter * 32 + lane;
    const bool odd = lane & 1;
    long long chunk = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
      int mt, nt, split, h, kb0, nkb;
      decode(t, &mt, &nt, &split, &h, &kb0, &nkb);
      const int nchunks = (nkb + P.chunk_kb - 1) / P.chunk_kb;
      const int grow = mt * TC_BM + row;  // row of A' within the batch
      const int m = grow >> 1;
      const size_t cbase = (size_t(h) * P.M + m) * size_t(P.N);
      float acc[128];
#pragma unroll
      for (int j = 0; j < 128; ++j) acc[j] = 0.f;
      for (int c = 0; c < nchunks; ++c, ++chunk) {
        const int b = int(chunk & 1);
        ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_full[b]), uint32_t(chunk >> 1) & 1));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (q < nq) {
            uint32_t v[32];
            TC_LD32(tmem + lane_addr + uint32_t(b) * buf_cols + uint32_t((q0 + q) * 32), v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[q * 32 + j] += __uint_as_float(v[j]);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
      }
      if (!ok) {
        if (lane == 0) atomicOr(P.err, 1);
        break;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (q >= nq) break;
        float re[16], im[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float mine_lo = acc[q * 32 + j], mine_hi = acc[q * 32 + 16 + j];
          const float other = __shfl_xor_sync(0xffffffffu, odd ? mine_lo : mine_hi, 1);
          // even lane (re row) keeps columns 0..15, odd lane (im row) keeps 16..31
          re[j] = odd ? other : mine_lo;
          im[j] = odd ? mine_hi : other;
        }
        if (m < P.M) {
          const int n0 = nt * P.BN + (q0 + q) * 32 + (odd ? 16 : 0);
          if (P.part) {
            float2* dst = P.part + size_t(split) * P.batch * P.M * P.N + cbase;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (n0 + j < P.N) dst[n0 + j] = make_float2(re[j], im[j]);
          } else if (P.acc) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (n0 + j < P.N) {
                double2 tt = P.acc[cbase + n0 + j];
                tt.x += double(re[j]);
                tt.y += double(im[j]);
                P.acc[cbase + n0 + j] = tt;
              }
          } else if (n0 + 16 <= P.N) {
            float4* dst = reinterpret_cast<float4*>(P.C + cbase + n0);
#pragma unroll
            for (int j = 0; j < 8; ++j) dst[j] = make_float4(re[2 * j], im[2 * j], re[2 * j + 1], im[2 * j + 1]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (n0 + j < P.N) P.C[cbase + n0 + j] = make_float2(re[j], im[j]);
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    // all MMAs of this CTA have completed before the accumulators are released
    if (!mbar_wait(smem_u32(&final_bar), 0) && lane == 0) atomicOr(P.err, 1);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 3D map over [batch][rows][inner] with a 128-byte swizzled box {inner_box, box_rows, 1}.
bool make_map(CUtensorMap* m, const void* base, bool bf16, uint64_t inner, uint64_t rows, uint64_t batch,
              uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const uint64_t es = bf16 ? 2 : 4;
  cuuint64_t dims[3] = {inner, rows, batch};
  cuuint64_t strides[2] = {inner * es, inner * rows * es};
  cuuint32_t box[3] = {uint32_t(128 / es), box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

cudaError_t tc_gemm_prepare() {
  // one-time set-up outside any stream capture: the driver entry point and the
  // largest dynamic shared memory any configuration of the kernel uses
  static cudaError_t result = cudaErrorUnknown;
  static std::once_flag once;
  std::call_once(once, [] {
    result = encode_fn() ? cudaSuccess : cudaErrorNotSupported;
    if (result == cudaSuccess)
      result = cudaFuncSetAttribute(cgemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BUDGET + 1024);
    if (result == cudaSuccess) result = tc_rows_prepare();
  });
  return result;
}

bool tc_gemm_supported(int M, int N, int K, int precision) {
  if (precision == TNQ_PREC_FP32) return false;
  const bool bf16 = precision == TNQ_PREC_BF16X3;
  // rows of 2K reals must be a multiple of 16 bytes and cover at least one MMA K step
  if (bf16 ? K < 8 : K < 4) return false;
  return M >= 1 && N >= 1;
}

cudaError_t launch_cgemm_tc(const TcGemmArgs& g, int sm_count, cudaStream_t st) {
  if (!tc_gemm_supported(g.M, g.N, g.K, g.precision) || !g.err) return cudaErrorNotSupported;
  const bool bf16 = g.precision == TNQ_PREC_BF16X3;
  const bool split = g.precision != TNQ_PREC_TF32;
  // each epilogue thread keeps at most 128 FP32 accumulator registers (BN/2 columns)
  int BN = 256;
  while (BN > 32 && BN / 2 >= g.N) BN /= 2;
  TcParams P;
  P.M = g.M;
  P.N = g.N;
  const uint64_t inner = 2ull * g.K;  // reals per row
  const int k_elems = bf16 ? 64 : 32;
  P.nkb = int((inner + k_elems - 1) / k_elems);
  P.tiles_m = int((2ull * g.M + TC_BM - 1) / TC_BM);
  P.tiles_n = (g.N + BN - 1) / BN;
  P.BN = BN;
  P.split = split ? 1 : 0;
  P.kind_bf16 = bf16 ? 1 : 0;
  P.a_bytes = TC_BM * TC_ROW_BYTES;
  P.b_bytes = uint32_t(BN) * TC_ROW_BYTES;
  const uint32_t stage_bytes = (split ? 2u : 1u) * (P.a_bytes + P.b_bytes);
  P.stages = std::min<int>(TC_MAX_STAGES, TC_SMEM_BUDGET / int(stage_bytes));
  if (P.stages < 2) return cudaErrorNotSupported;
  P.stage_tx = stage_bytes;
  P.chunk_kb = split ? 2 : (1 << 30);  // non-split modes: one chunk per tile
  // instruction descriptor: FP32 accumulator, A/B format (TF32 = 2, BF16 = 1), K-major, N >> 3, M >> 4
  const uint32_t fmt = bf16 ? 1u : 2u;
  P.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(TC_BM >> 4) << 24);
  P.C = reinterpret_cast<float2*>(g.c);
  P.acc = reinterpret_cast<double2*>(g.acc);
  P.err = g.err;
  P.batch = g.batch;
  P.splits = std::max(1, std::min(g.splits, P.nkb));
  P.kb_per_split = (P.nkb + P.splits - 1) / P.splits;
  P.splits = (P.nkb + P.kb_per_split - 1) / P.kb_per_split;  // every split owns >= 1 K block
  P.part = P.splits > 1 ? reinterpret_cast<float2*>(g.part) : nullptr;
  if (P.splits > 1 && !g.part) return cudaErrorInvalidValue;
  const long long total = (long long)P.tiles_m * P.tiles_n * P.splits * g.batch;
  if (total > 0x7fffffffLL) return cudaErrorNotSupported;
  CUtensorMap ma_hi, ma_lo, mb_hi, mb_lo;
  if (!make_map(&ma_hi, g.a_hi, bf16, inner, 2ull * g.M, g.batch, TC_BM)) return cudaErrorInvalidValue;
  if (!make_map(&mb_hi, g.b_hi, bf16, inner, g.N, g.batch, BN)) return cudaErrorInvalidValue;
  if (split) {
    if (!make_map(&ma_lo, g.a_lo, bf16, inner, 2ull * g.M, g.batch, TC_BM)) return cudaErrorInvalidValue;
    if (!make_map(&mb_lo, g.b_lo, bf16, inner, g.N, g.batch, BN)) return cudaErrorInvalidValue;
  } else {
    ma_lo = ma_hi;
    mb_lo = mb_hi;
  }
  const int smem = int(P.stages * stage_bytes) + 1024;
  cudaError_t pe = tc_gemm_prepare();
  if (pe != cudaSuccess) return pe;
  // Short-K tiles: persistent CTAs (one per SM) loop over their tiles so the
  // next tile's loads and MMAs overlap this tile's epilogue.  Long-K tiles:
  // one CTA per tile (the loop runs once), which measured faster there.
  const long long grid = P.kb_per_split <= 16 ? std::min<long long>(total, std::max(1, sm_count)) : total;
  cgemm_tc_kernel<<<unsigned(grid), TC_THREADS, smem, st>>>(ma_hi, ma_lo, mb_hi, mb_lo, P);
  if (g.splits_used) *g.splits_used = P.splits;
  return cudaGetLastError();
}

}  // namespace tnq
