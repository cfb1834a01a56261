// Tall-skinny complex GEMM on the tcgen05 tensor cores, sm_103a.
//
// Steps of the contraction sequence (Sec. 3.1) whose one operand is small
// (ns <= 128 rows) and whose contracted extent is short (K <= 256) but whose
// other operand G is large (ng rows, up to 2^24 and more) do 8 * ns real flops
// per byte of G: too few for a tensor-core tile built the ordinary way (the
// 2 * ns-row expansion of the small operand would fill part of a 128-row MMA
// and the large operand would need a permute and a separate hi/lo split), too
// many for the CUDA cores to keep up with HBM.  Here the roles are swapped:
// 128 rows of G form the MMA's M side, the expanded small operand
//   S' (2 ns x 2K):  row (s, re) = [sr_0, -si_0, sr_1, -si_1, ...]
//                    row (s, im) = [si_0,  sr_0, si_1,  sr_1, ...]
// its N side, and D = G * S'^T leaves Re/Im of out[s][g] in TMEM columns
// (2s, 2s+1) of lane g.
//
// G is read once from HBM, in its stored bit order (the gather of the permute
// is fused: the row and K bits of G sit at arbitrary positions of the stored
// tensor), split into hi/lo parts (BF16 or TF32) by converter warps and written
// straight into the 128-byte-swizzled K-major layout the MMA reads (128-byte
// swizzle atoms of K per row).  The output is written once.  Per 128-row
// tile: 128 * K * 8 bytes in, 128 * ns * 8 bytes out, 2 * ceil(2K / k_step)
// MMAs in the split modes (Npad = max(16, 2 ns) <= 128: one of 128 x 2 Npad
// over S' hi and lo rows side by side, one of 128 x Npad; three of 128 x Npad
// for Npad = 256), ceil(2K / k_step) in plain TF32; four TMEM accumulator
// buffers for Npad <= 64, two above, at most all 512 columns.  When the
// expanded small operand of every batch entry does not fit in shared memory,
// each batch entry gets its own launch.
//
// A tile's K range may be cut into one-atom K-parts: a shared-memory stage
// then holds one part of a tile (the MMAs of a tile accumulate over its
// parts), which lets TF32 rows of K = 64 (four atoms) run in three stages
// beside a 128 KB expanded small operand.  Rows of K = 128 or 256 stream the
// expanded small operand as well: it is built once in global memory (where it
// stays in L2) and each stage receives the K-part of it that its MMAs read, by
// a bulk copy that completes on the stage's barrier.
//
// In the split modes the product hi*hi accumulates into one TMEM buffer and
// the two correction products hi*lo, lo*hi into a second one beside it (hi*hi
// and hi*lo are one MMA); the epilogue adds them in FP32 registers.  The
// tensor-memory accumulator adds each MMA's result with truncation toward
// zero, so a chain of additions into the large accumulator shrinks it by about
// half an ulp per addition; keeping the corrections (about 2^-9 of it) apart
// cuts that chain to one addition per K step.
//
// CTA (persistent; one per SM, or two where the stages, S' and TMEM buffers
// fit in half an SM) = 13 warps:
//   warps 0-7   converters, two groups of four; group g fills the stages of
//               the CTA's items i = g, g + 2, ... (an item is one K-part of a
//               tile): each thread owns one tile row and walks the item's K
//               range in chunks of up to 16 complex values (loads
//               of 16-byte pairs when the lowest stored bit is a K bit); the
//               loads of the next chunks are issued before the current one is
//               split and stored, and the register ring rotates by moves,
//               which wait for the newest load, so in effect one chunk is in
//               flight across each split (an unrolled ring without the moves
//               measured slower);
//   warp 8      allocates TMEM and (one thread) issues the MMAs of each tile
//               into one of the TMEM accumulator buffers;
//   warps 9-12  epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, 32
//               columns at a time (16 with two CTAs per SM), and the
//               correction buffer's columns, the next columns' loads in
//               flight while it writes complex64 outputs (or adds into the
//               FP64 cross-slice sum).
// Every mbarrier wait is bounded; one that runs out sets the error flag and
// the CTA unwinds.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "gemm_tc.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"
#include "../../include/tnq.h"

namespace tnq {

namespace {

using namespace tcx;

constexpr int TR_CONV_WARPS = 8;
constexpr int TR_THREADS = 32 * (TR_CONV_WARPS + 1 + 4);
constexpr int TR_MMA_WARP = TR_CONV_WARPS;
constexpr int TR_MAX_STAGES = 4;
constexpr int TR_MAX_NACC = 4;                 // TMEM accumulator buffers
constexpr int TR_ROW_BYTES = 128;              // one swizzle atom of a row
constexpr int TR_ATOM_BYTES = 128 * TR_ROW_BYTES;  // one atom column of a 128-row tile
constexpr int TR_BPRIME_BUDGET = 128 * 1024;
constexpr int TR_SMEM_LIMIT = 225 * 1024;      // dynamic shared memory of one CTA
constexpr int TR_SMEM_HALF = 110 * 1024;       // the same, two CTAs per SM
constexpr int TR_KMAX = 256;                  // longest K (in resident mode: 64)
constexpr int TR_ROWTAB_DIGITS = 7;           // 4-bit digits of a tile index (nrow <= 35)

struct TrParams {
  const float2* S;        // small operand [batch][ns][K]
  const float2* G;        // large operand, stored bit order (see gd)
  GatherDesc gd;          // rows: g bits then batch bits; K bits in contraction order
  int ns, ng, K, batch;
  int npad;               // MMA N: max(16, 2 ns)
  int nks;                // MMA K steps (32 bytes of K per step) of a whole row
  int atoms;              // 128-byte swizzle atoms per row (1 to 4)
  int kparts;             // K-parts per tile (items per tile)
  int patoms;             // atoms per part: atoms / kparts
  int nks_part;           // MMA K steps per part
  int kc;                 // complex values per part
  int stages;             // shared-memory stages, each holding one part
  int nacc;               // TMEM accumulator buffers
  int dual;               // 1: correction products in a second TMEM buffer
  int merged;             // 1 (dual): hi*hi and hi*lo in one MMA of N = 2 npad over S' hi and lo rows
  int acc_cols;           // TMEM columns per accumulator buffer: npad, or 2 npad when dual
  int nchunks;            // converter chunks per part
  int stream_bp;          // 1: S' streamed per K-part from bp_glob into each stage (long K)
  const uint8_t* bp_glob; // streamed mode: S' expanded in global memory, same layout as in shared memory
  uint32_t bp_part;       // streamed mode: bytes of S' hi (or lo) rows for one K-part
  int kind_bf16;          // 1: BF16 parts, kind::f16; 0: TF32 parts, kind::tf32
  int split;              // 1: three products (hi/lo); 0: one TF32 product
  int pairs;              // the lowest stored bit of G is K bit 0: 16-byte loads
  int row_tab;            // 1: every stored position of the row bits above 7 is below 32 (digit table)
  long long s_stride, g_stride;
  int tiles_per_h;        // ng / 128
  long long total_tiles;
  int slice_id;
  uint32_t idesc;         // MMA of N = npad
  uint32_t idesc2;        // MMA of N = 2 npad (merged)
  float2* C;
  double2* acc;
  int* err;
};

__device__ __forceinline__ uint32_t bf16_bits(float x) {
  return uint32_t(__bfloat16_as_ushort(__float2bfloat16_rn(x)));
}

__device__ __forceinline__ float bf16_val(uint32_t b) { return __uint_as_float(b << 16); }

// Nearest TF32 value (10 stored mantissa bits), ties away from zero: half a
// unit of the last kept bit is added to the magnitude field and the 13
// dropped bits are cleared (a carry into the exponent gives the next binade,
// or infinity past the largest finite value, as the rounding requires).
// Integer operations on the full-rate ALU pipe; finite inputs.
__device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

// hi/lo words of two reals (x0, x1) packed for one 4-byte slot of a BF16 row.
__device__ __forceinline__ void bf16_split2(float x0, float x1, uint32_t* hi, uint32_t* lo) {
  const uint32_t h0 = bf16_bits(x0), h1 = bf16_bits(x1);
  const uint32_t l0 = bf16_bits(x0 - bf16_val(h0)), l1 = bf16_bits(x1 - bf16_val(h1));
  *hi = h0 | (h1 << 16);
  *lo = l0 | (l1 << 16);
}

// Byte offset of 16-byte unit u of row r in a K-major tile of 128-byte-swizzled
// atoms: atom u / 8 (atom columns atom_bytes apart), 8-row groups of 1024 bytes
// within an atom, unit index XOR row-in-group.
__device__ __forceinline__ uint32_t swz(int r, int u, uint32_t atom_bytes) {
  return uint32_t(u >> 3) * atom_bytes + uint32_t(r) * 128u + (uint32_t((u & 7) ^ (r & 7)) << 4);
}

// Split chunk c (complex values c*CH .. c*CH+CH-1 of the row, zero beyond K)
// and store its 16-byte units that the MMAs read (units < 2 * nks).
template <int CH>
__device__ __forceinline__ void store_chunk(uint8_t* hi, uint8_t* lo, int r, const float2 (&v)[CH], int c,
                                            int units, int kind_bf16, int split) {
  if (kind_bf16) {
    // one unit: 4 complex values (8 BF16 reals)
#pragma unroll
    for (int j = 0; j < CH / 4; ++j) {
      const int u = c * (CH / 4) + j;
      if (u < units) {
        uint4 h, l;
        bf16_split2(v[4 * j].x, v[4 * j].y, &h.x, &l.x);
        bf16_split2(v[4 * j + 1].x, v[4 * j + 1].y, &h.y, &l.y);
        bf16_split2(v[4 * j + 2].x, v[4 * j + 2].y, &h.z, &l.z);
        bf16_split2(v[4 * j + 3].x, v[4 * j + 3].y, &h.w, &l.w);
        *reinterpret_cast<uint4*>(hi + swz(r, u, TR_ATOM_BYTES)) = h;
        *reinterpret_cast<uint4*>(lo + swz(r, u, TR_ATOM_BYTES)) = l;
      }
    }
  } else {
    // one unit: 2 complex values (4 TF32 reals)
#pragma unroll
    for (int j = 0; j < CH / 2; ++j) {
      const int u = c * (CH / 2) + j;
      if (u < units) {
        float4 h, l;
        h.x = tf32_rna(v[2 * j].x);
        h.y = tf32_rna(v[2 * j].y);
        h.z = tf32_rna(v[2 * j + 1].x);
        h.w = tf32_rna(v[2 * j + 1].y);
        *reinterpret_cast<float4*>(hi + swz(r, u, TR_ATOM_BYTES)) = h;
        if (split) {
          l.x = tf32_rna(v[2 * j].x - h.x);
          l.y = tf32_rna(v[2 * j].y - h.y);
          l.z = tf32_rna(v[2 * j + 1].x - h.z);
          l.w = tf32_rna(v[2 * j + 1].y - h.w);
          *reinterpret_cast<float4*>(lo + swz(r, u, TR_ATOM_BYTES)) = l;
        }
      }
    }
  }
}

// Expanded small operand S' for every batch entry: rows n < npad of the reals
// the MMAs read, hi and lo, built by the converter threads at kernel start.
__device__ void build_bprime(const TrParams& P, uint8_t* bp, int tid, int nthreads) {
  const int es = P.kind_bf16 ? 2 : 4;
  const int reals = P.nks * (32 / es);
  const int per_h = P.npad * reals;
  // per batch entry and atom column: npad hi rows, then npad lo rows
  const uint32_t atom_bytes = 2u * uint32_t(P.npad) * TR_ROW_BYTES;
  const uint32_t entry_bytes = atom_bytes * P.atoms;
  for (int e = tid; e < P.batch * per_h; e += nthreads) {
    const int h = e / per_h, rem = e % per_h, n = rem / reals, q = rem % reals;
    const int s = n >> 1, k = q >> 1;
    float x = 0.f;
    if (s < P.ns && k < P.K) {
      const float2 a = P.S[(size_t(h) * P.ns + s) * P.K + k];
      // row (s, re): [sr, -si] per k; row (s, im): [si, sr]
      x = (n & 1) ? ((q & 1) ? a.x : a.y) : ((q & 1) ? -a.y : a.x);
    }
    uint8_t* hi = bp + size_t(h) * entry_bytes;
    uint8_t* lo = hi + uint32_t(P.npad) * TR_ROW_BYTES;  // row npad + n: same swizzle phase (npad % 16 == 0)
    const uint32_t off = swz(n, (q * es) >> 4, atom_bytes) + uint32_t((q * es) & 15);
    if (P.kind_bf16) {
      const uint32_t hb = bf16_bits(x);
      *reinterpret_cast<unsigned short*>(hi + off) = (unsigned short)hb;
      *reinterpret_cast<unsigned short*>(lo + off) = (unsigned short)bf16_bits(x - bf16_val(hb));
    } else {
      const float hv = tf32_rna(x);
      *reinterpret_cast<float*>(hi + off) = hv;
      *reinterpret_cast<float*>(lo + off) = tf32_rna(x - hv);
    }
  }
}

// S' of every batch entry expanded into global memory (streamed mode), in the
// layout build_bprime gives it in shared memory.
__global__ void build_bprime_kernel(const __grid_constant__ TrParams P, uint8_t* dst) {
  build_bprime(P, dst, int(blockIdx.x * blockDim.x + threadIdx.x), int(gridDim.x * blockDim.x));
}

// Tile t = h * tph + gt (batch entry h, tile gt within it), stepped by the
// grid stride without a division in the common case (stride < 2 tph).
struct TileHG {
  uint32_t h, gt;
};

__device__ __forceinline__ TileHG tile_hg(uint32_t t, uint32_t tph) {
  const uint32_t h = t / tph;
  return TileHG{h, t - h * tph};
}

__device__ __forceinline__ void tile_step(TileHG& q, uint32_t step, uint32_t tph) {
  q.gt += step;
  if (q.gt >= tph) {
    if (q.gt < 2 * tph) {
      q.gt -= tph;
      ++q.h;
    } else {
      q.h += q.gt / tph;
      q.gt %= tph;
    }
  }
}

__device__ __forceinline__ size_t deposit(long long v, const int* pos, int n) {
  size_t o = 0;
  for (int j = 0; j < n; ++j)
    if ((v >> j) & 1) o |= size_t(1) << pos[j];
  return o;
}

// Chunk c of K-part kp of the row whose K = 0 element sits at stored offset `base`.
template <int CH>
__device__ __forceinline__ void load_chunk(const TrParams& P, const uint32_t* koff, size_t base, int kp, int c,
                                           float2 (&v)[CH]) {
  const int k0 = kp * P.kc + c * CH;
  if (P.pairs) {
#pragma unroll
    for (int j = 0; j < CH; j += 2) {
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k0 + j < P.K) t = __ldg(reinterpret_cast<const float4*>(P.G + base + koff[k0 + j]));
      v[j] = make_float2(t.x, t.y);
      v[j + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int j = 0; j < CH; ++j) v[j] = k0 + j < P.K ? __ldg(P.G + base + koff[k0 + j]) : make_float2(0.f, 0.f);
  }
}

// MODE: 0 plain TF32, 1 TF32x3, 2 BF16x3.  The converter loop is unrolled,
// and a kernel holding every mode's conversion code made the rarely running
// MMA warp miss in the instruction cache (about 200 cycles per group of
// instructions it issued), so each mode is its own kernel.
// MINB: CTAs per SM (2 for launches whose stages, S' and TMEM buffers fit in
// half an SM: twice the warps to hide the roles' latencies, 72 registers).
template <int CH, int DEPTH, int MODE, int MINB>
__global__ void __launch_bounds__(TR_THREADS, MINB) cgemm_tc_rows_kernel(const __grid_constant__ TrParams P) {
  extern __shared__ uint8_t smem_raw[];
  constexpr int kBF16 = MODE == 2 ? 1 : 0, kSplit = MODE != 0 ? 1 : 0;
  __shared__ __align__(8) uint64_t full_bar[TR_MAX_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[TR_MAX_STAGES];
  __shared__ __align__(8) uint64_t acc_full[TR_MAX_NACC];
  __shared__ __align__(8) uint64_t acc_empty[TR_MAX_NACC];
  __shared__ __align__(8) uint64_t final_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ uint32_t koff[TR_KMAX];
  // deposit of each 4-bit digit of a tile index into the stored positions of
  // the row bits above the lowest 7 (used when every position is below 32)
  __shared__ uint32_t rowtab[TR_ROWTAB_DIGITS][16];

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // a stage: G hi and lo of one K-part, then (streamed mode) S' hi and lo of that part
  const uint32_t g_piece = TR_ATOM_BYTES * uint32_t(P.patoms);
  const uint32_t stage_bytes = 2u * g_piece + (P.stream_bp ? 2u * P.bp_part : 0u);
  uint8_t* bprime = smem + size_t(P.stages) * stage_bytes;
  const uint32_t bp_atom = 2u * uint32_t(P.npad) * TR_ROW_BYTES;  // S' hi and lo rows of one atom column
  const uint32_t bp_entry = bp_atom * uint32_t(P.atoms);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tmem_cols = uint32_t(P.acc_cols * P.nacc) < 32u ? 32u : uint32_t(P.acc_cols * P.nacc);

  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) {
      // one converter group, plus the transaction arrival of the S' copy
      mbar_init(smem_u32(&full_bar[s]), 128 + (P.stream_bp ? 1 : 0));
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < P.nacc; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), 4);  // one arrival per epilogue warp
    }
    mbar_init(smem_u32(&final_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int kk = threadIdx.x; kk < TR_KMAX; kk += blockDim.x) {
    uint32_t o = 0;
    for (int j = 0; j < P.gd.nk; ++j)
      if ((kk >> j) & 1) o |= 1u << P.gd.kpos[j];
    koff[kk] = o;
  }
  const int nhi_all = P.gd.nrow - 7, ndig = (nhi_all + 3) / 4;
  const bool use_rowtab = P.row_tab != 0;
  if (use_rowtab)
    for (int e = threadIdx.x; e < ndig * 16; e += blockDim.x) {
      const int n = e >> 4, v = e & 15;
      uint32_t o = 0;
      for (int b = 0; b < 4 && 4 * n + b < nhi_all; ++b)
        if ((v >> b) & 1) o |= 1u << P.gd.rowpos[7 + 4 * n + b];
      rowtab[n][v] = o;
    }
  if (warp < TR_CONV_WARPS && !P.stream_bp) build_bprime(P, bprime, threadIdx.x, 32 * TR_CONV_WARPS);
  if (warp == TR_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  // S' written by generic stores becomes visible to the MMA (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t tph = uint32_t(P.tiles_per_h), total = uint32_t(P.total_tiles);
  const int kparts = P.kparts;

  if (warp < TR_CONV_WARPS) {
    // ---------------- converters: group grp fills the stages of items grp, grp+2, ...
    // CTA-local item j is K-part j % kparts of the CTA's tile j / kparts
    // (global tile blockIdx.x + (j / kparts) * gridDim.x); it uses stage
    // j % stages, phase (j / stages) & 1.  The cursors below carry these
    // quotients and remainders from item to item instead of dividing.
    const int grp = warp >> 2, r = (warp & 3) * 32 + lane;
    const int nhi = P.gd.nrow - 7;
    const int nch = P.nchunks, units = 2 * P.nks_part;
    const uint32_t nst = uint32_t(P.stages);
    size_t soff = 0;
    for (int j = 0; j < P.gd.n_slice; ++j)
      if (P.gd.slice_src[j] >= 0 && ((P.slice_id >> j) & 1)) soff |= size_t(1) << P.gd.slice_src[j];
    const size_t lo = soff | deposit(r, P.gd.rowpos, 7);
    // row r of tile t is row 128 t + r of the (batch-major) row index, whose
    // bits above the lowest 7 are t itself
    auto row_base = [&](uint32_t t) {
      if (!use_rowtab) return lo | deposit((long long)t, P.gd.rowpos + 7, nhi);
      size_t o = lo;
      for (int n = 0; n < ndig; ++n) o |= rowtab[n][(t >> (4 * n)) & 15u];
      return o;
    };
    // item cursor: K-part and tile of item j, advanced by the group stride 2
    struct ItemCursor {
      uint32_t kp, tile;
    };
    auto first_item = [&]() {
      ItemCursor q{uint32_t(grp), blockIdx.x};
      while (q.kp >= uint32_t(kparts)) {
        q.kp -= uint32_t(kparts);
        q.tile += gridDim.x;
      }
      return q;
    };
    auto next_item = [&](ItemCursor& q) {
      q.kp += 2;
      while (q.kp >= uint32_t(kparts)) {
        q.kp -= uint32_t(kparts);
        q.tile += gridDim.x;
      }
    };
    // items (item, chunk c) in order: the loads of the next DEPTH chunks are in
    // flight while one is split and stored.
    ItemCursor ql = first_item();  // load cursor: item, chunk, its tile's row base
    int cl = 0;
    size_t bl = ql.tile < total ? row_base(ql.tile) : 0;
    auto advance_load = [&]() {
      if (++cl == nch) {
        cl = 0;
        const uint32_t t0 = ql.tile;
        next_item(ql);
        if (ql.tile != t0) bl = ql.tile < total ? row_base(ql.tile) : 0;
      }
    };
    float2 buf[DEPTH + 1][CH];
#pragma unroll
    for (int d = 0; d < DEPTH; ++d) {
      if (ql.tile < total) load_chunk<CH>(P, koff, bl, int(ql.kp), cl, buf[d]);
      advance_load();
    }
    ItemCursor qc = first_item();  // convert cursor
    uint32_t s = uint32_t(grp), ph = 0;  // its stage and phase: j % stages, (j / stages) & 1
    int c = 0;
    while (qc.tile < total) {
      // the empty wait orders this item after the MMAs of item j - stages,
      // whichever group converted that one, so any stage count works
      if (ql.tile < total) load_chunk<CH>(P, koff, bl, int(ql.kp), cl, buf[DEPTH]);
      advance_load();
      if (c == 0 && !mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1)) {
        atomicOr(P.err, 1);
        break;
      }
      uint8_t* st = smem + size_t(s) * stage_bytes;
      if (c == 0 && P.stream_bp && r == 0) {
        // S' hi and lo of this item's K-part, copied into the stage by the bulk
        // copy engine; the stage completes when both copies have landed
        const uint8_t* src = P.bp_glob + size_t(qc.tile / tph) * bp_entry + size_t(qc.kp) * 2u * P.bp_part;
        const uint32_t bar = smem_u32(&full_bar[s]);
        mbar_expect_tx(bar, 2u * P.bp_part);
        bulk_g2s(smem_u32(st + 2 * g_piece), src, 2u * P.bp_part, bar);
      }
      store_chunk<CH>(st, st + g_piece, r, buf[0], c, units, kBF16, kSplit);
      if (c == nch - 1) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&full_bar[s]));
      }
#pragma unroll
      for (int d = 0; d < DEPTH; ++d)
#pragma unroll
        for (int j = 0; j < CH; ++j) buf[d][j] = buf[d + 1][j];
      if (++c == nch) {
        c = 0;
        next_item(qc);
        s += 2;
        while (s >= nst) {
          s -= nst;
          ph ^= 1u;
        }
      }
    }
  } else if (warp == TR_MMA_WARP) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int s = 0, b = 0;
      uint32_t sph = 0, bph = 0;  // phases of the stage ring and of the accumulator ring
      bool drained = false;       // every accumulator buffer has been used once
      bool ok = true;
      TileHG hg = tile_hg(blockIdx.x, tph);
      for (uint32_t t = blockIdx.x; t < total && ok; t += gridDim.x, tile_step(hg, gridDim.x, tph)) {
        if (drained && !mbar_wait(smem_u32(&acc_empty[b]), bph ^ 1)) {
          atomicOr(P.err, 1);
          break;
        }
        const uint32_t h = hg.h;
        const uint32_t d = tmem + uint32_t(b * P.acc_cols);
        const uint32_t dc = P.dual ? d + uint32_t(P.npad) : d;  // correction products
        for (int kp = 0; kp < kparts; ++kp) {
          if (!mbar_wait(smem_u32(&full_bar[s]), sph)) {
            atomicOr(P.err, 1);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a_hi = smem_u32(smem + size_t(s) * stage_bytes), a_lo = a_hi + g_piece;
          // S': this part in the stage (streamed) or the whole row resident
          const uint32_t b_hi = P.stream_bp ? a_hi + 2 * g_piece : smem_u32(bprime) + h * bp_entry;
          // shared-memory addresses stay below 2^18, so a descriptor's address
          // field (address >> 4) takes byte offsets >> 4 without carrying out
          const uint64_t da_hi = smem_desc(a_hi), da_lo = smem_desc(a_lo), db_hi = smem_desc(b_hi);
          const uint64_t db_lo = db_hi + uint64_t((uint32_t(P.npad) * TR_ROW_BYTES) >> 4);
          for (int kk = 0; kk < P.nks_part; ++kk) {
            const int kg = kp * P.nks_part + kk;  // K step within the row
            const uint64_t ao = uint64_t((uint32_t(kk >> 2) * TR_ATOM_BYTES + uint32_t(kk & 3) * 32) >> 4);
            const int kb = P.stream_bp ? kk : kg;  // K step within the S' buffer the MMA reads
            const uint64_t bo = uint64_t((uint32_t(kb >> 2) * bp_atom + uint32_t(kb & 3) * 32) >> 4);
            const uint32_t acc_on = kg > 0 ? 1u : 0u;
            if (P.merged) {
              // columns [0, npad): hi*hi; [npad, 2 npad): hi*lo, then lo*hi added
              mma_issue(kBF16, d, da_hi + ao, db_hi + bo, P.idesc2, acc_on);
              mma_issue(kBF16, dc, da_lo + ao, db_hi + bo, P.idesc, 1u);
            } else if (kSplit) {
              mma_issue(kBF16, dc, da_lo + ao, db_hi + bo, P.idesc, acc_on);
              mma_issue(kBF16, dc, da_hi + ao, db_lo + bo, P.idesc, 1u);
              mma_issue(kBF16, d, da_hi + ao, db_hi + bo, P.idesc, P.dual ? acc_on : 1u);
            } else {
              mma_issue(kBF16, d, da_hi + ao, db_hi + bo, P.idesc, acc_on);
            }
          }
          mma_commit(smem_u32(&empty_bar[s]));
          if (++s == P.stages) {
            s = 0;
            sph ^= 1;
          }
        }
        if (!ok) break;
        mma_commit(smem_u32(&acc_full[b]));
        if (++b == P.nacc) {
          b = 0;
          bph ^= 1;
          drained = true;
        }
      }
      mma_commit(smem_u32(&final_bar));
    }
    __syncwarp();
  } else {
    // ---------------- epilogue
    const int quarter = warp & 3;
    const uint32_t lane_addr = uint32_t(quarter * 32) << 16;
    const int row = quarter * 32 + lane;
    int b = 0;
    uint32_t bph = 0;
    TileHG hg = tile_hg(blockIdx.x, tph);
    for (uint32_t t = blockIdx.x; t < total; t += gridDim.x, tile_step(hg, gridDim.x, tph)) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_full[b]), bph));
      if (!ok) {
        if (lane == 0) atomicOr(P.err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t h = hg.h;
      const uint32_t g = hg.gt * 128u + uint32_t(row);
      const size_t obase = size_t(h) * P.ns * P.ng + size_t(g) * P.g_stride;
      const uint32_t base = tmem + lane_addr + uint32_t(b * P.acc_cols);
      // 32 columns (16 outputs) at a time
      // EC columns (EC / 2 outputs) at a time; the TMEM loads of the next EC
      // columns are in flight while this group is stored, and the buffer is
      // released as soon as its last columns are in registers
      constexpr int EC = MINB == 2 ? 16 : 32;
      uint32_t v[EC], w[EC];
      auto tmem_ld = [&](int c0) {
        TC_LD16(base + c0, v);
        if constexpr (EC == 32)
          if (c0 + 16 < P.npad) TC_LD16(base + c0 + 16, (v + 16));
        if (P.dual) {
          TC_LD16(base + P.npad + c0, w);
          if constexpr (EC == 32)
            if (c0 + 16 < P.npad) TC_LD16(base + P.npad + c0 + 16, (w + 16));
        }
      };
      tmem_ld(0);
      for (int c0 = 0; c0 < P.npad; c0 += EC) {
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if constexpr (EC == 32) {
          TC_PIN32(v);
          TC_PIN32(w);
        } else {
          TC_PIN16(v);
          TC_PIN16(w);
        }
        float o[EC];
#pragma unroll
        for (int j = 0; j < EC; ++j) o[j] = P.dual ? __uint_as_float(v[j]) + __uint_as_float(w[j]) : __uint_as_float(v[j]);
        if (c0 + EC < P.npad) {
          tmem_ld(c0 + EC);
        } else {
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
        }
#pragma unroll
        for (int j = 0; j < EC / 2; ++j) {
          const int s = c0 / 2 + j;
          if (s < P.ns) {
            const float re = o[2 * j], im = o[2 * j + 1];
            const size_t o_at = obase + size_t(s) * P.s_stride;
            if (P.acc) {
              double2 a = P.acc[o_at];
              a.x += double(re);
              a.y += double(im);
              P.acc[o_at] = a;
            } else {
              P.C[o_at] = make_float2(re, im);
            }
          }
        }
      }
      if (++b == P.nacc) {
        b = 0;
        bph ^= 1;
      }
    }
  }
  __syncthreads();
  if (warp == TR_MMA_WARP) {
    // every MMA of this CTA has completed before TMEM is released
    if (!mbar_wait(smem_u32(&final_bar), 0) && lane == 0) atomicOr(P.err, 1);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

}  // namespace

// ---------------------------------------------------------------- host side
namespace {

int tr_npad(int ns) { return std::max(16, (2 * ns + 15) / 16 * 16); }

// 128-byte swizzle atoms per row: 2K reals of 2 (BF16) or 4 (TF32) bytes
int tr_atoms(int K, bool bf16) { return (2 * K * (bf16 ? 2 : 4) + TR_ROW_BYTES - 1) / TR_ROW_BYTES; }

size_t tr_bprime_bytes(int ns, int K, int batch, bool bf16) {
  return size_t(batch) * 2 * tr_atoms(K, bf16) * tr_npad(ns) * TR_ROW_BYTES;
}

// Stage layout of a launch: K-parts per tile and stages.  A row of one or two
// atoms is one part (four stages with one atom, two with two); longer rows
// (TF32 with K = 64: four atoms) are cut into one-atom parts.  The stages plus
// the expanded small operand (bprime bytes) must fit the shared-memory limit.
struct TrStages {
  int kparts = 0, patoms = 0, stages = 0;
  bool stream = false;  // S' streamed per K-part (K > 64)
};

TrStages tr_stages(int atoms, size_t bprime) {
  TrStages t;
  if (atoms <= 2) {
    t.kparts = 1;
    t.patoms = atoms;
    t.stages = atoms == 1 ? 4 : 2;
  } else {
    t.kparts = atoms;
    t.patoms = 1;
    t.stages = 4;
  }
  const size_t stage_bytes = size_t(2) * TR_ATOM_BYTES * t.patoms;
  // one-atom parts may take an odd number of stages (three beside a 128 KB S')
  const int step = t.kparts > 1 ? 1 : 2;
  while (t.stages > 2 && size_t(t.stages) * stage_bytes + bprime + 1024 > size_t(TR_SMEM_LIMIT)) t.stages -= step;
  if (size_t(t.stages) * stage_bytes + bprime + 1024 > size_t(TR_SMEM_LIMIT)) t.stages = 0;
  return t;
}

// Streamed layout (K > 64): one-atom K-parts; a stage holds G hi and lo and
// the same part of S' hi and lo (npad rows of one atom each).
TrStages tr_stages_streamed(int atoms, int npad) {
  TrStages t;
  t.kparts = atoms;
  t.patoms = 1;
  t.stream = true;
  const size_t stage_bytes = size_t(2) * TR_ATOM_BYTES + size_t(2) * npad * TR_ROW_BYTES;
  t.stages = 4;
  while (t.stages > 2 && size_t(t.stages) * stage_bytes + 1024 > size_t(TR_SMEM_LIMIT)) t.stages -= 1;
  if (size_t(t.stages) * stage_bytes + 1024 > size_t(TR_SMEM_LIMIT)) t.stages = 0;
  return t;
}

constexpr size_t TR_SMEM_MAX = size_t(TR_SMEM_LIMIT);
constexpr int TR_RESIDENT_KMAX = 64;

}  // namespace

size_t tc_rows_scratch_bytes(int ns, int K, int batch, int precision) {
  if (K <= TR_RESIDENT_KMAX) return 0;
  return tr_bprime_bytes(ns, K, batch, precision == TNQ_PREC_BF16X3);
}

// kernels by [CH == 16][MODE]
using TrKernel = void (*)(TrParams);
const TrKernel kTrKernels[2][3] = {
    {cgemm_tc_rows_kernel<8, 4, 0, 1>, cgemm_tc_rows_kernel<8, 4, 1, 1>, cgemm_tc_rows_kernel<8, 4, 2, 1>},
    {cgemm_tc_rows_kernel<16, 2, 0, 1>, cgemm_tc_rows_kernel<16, 2, 1, 1>, cgemm_tc_rows_kernel<16, 2, 2, 1>},
};
// two CTAs per SM, by [MODE]
const TrKernel kTrKernels2[3] = {cgemm_tc_rows_kernel<8, 2, 0, 2>, cgemm_tc_rows_kernel<8, 2, 1, 2>,
                                 cgemm_tc_rows_kernel<8, 2, 2, 2>};


cudaError_t tc_rows_prepare() {
  static cudaError_t result = cudaErrorUnknown;
  static std::once_flag once;
  std::call_once(once, [] {
    result = cudaSuccess;
    for (const auto& row : kTrKernels)
      for (TrKernel k : row)
        if (result == cudaSuccess)
          result = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TR_SMEM_MAX));
    for (TrKernel k : kTrKernels2)
      if (result == cudaSuccess)
        result = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TR_SMEM_HALF));
  });
  return result;
}

bool tc_rows_supported(int ns, int ng, int K, int batch, int nrow, int precision) {
  if (precision != TNQ_PREC_TF32 && precision != TNQ_PREC_TF32X3 && precision != TNQ_PREC_BF16X3) return false;
  const bool bf16 = precision == TNQ_PREC_BF16X3;
  // MMA N = 2 ns <= 256; K up to 256 (rows of more than 64 complex values
  // stream S' through the stages)
  if (ns < 1 || ns > 128 || K < 1 || K > TR_KMAX || ng < 128 || (ng & 127) || batch < 1 || nrow < 7) return false;
  if (K > TR_RESIDENT_KMAX) return K >= 128 && tr_stages_streamed(tr_atoms(K, bf16), tr_npad(ns)).stages >= 2;
  // S' of one batch entry must fit beside at least two stages (larger batches
  // run one launch per entry)
  const size_t bp = tr_bprime_bytes(ns, K, 1, bf16);
  return bp <= size_t(TR_BPRIME_BUDGET) && tr_stages(tr_atoms(K, bf16), bp).stages >= 2;
}

namespace {

cudaError_t launch_tc_rows_one(const void* Ssmall, const void* Gsrc, const GatherDesc& gd, void* C, void* acc, int ns,
                               int ng, int K, int batch, long long s_stride_out, long long g_stride_out, int slice_id,
                               int precision, int* err, int sm_count, cudaStream_t st, void* scratch = nullptr,
                               size_t scratch_bytes = 0) {
  TrParams P;
  P.S = reinterpret_cast<const float2*>(Ssmall);
  P.G = reinterpret_cast<const float2*>(Gsrc);
  P.gd = gd;
  P.ns = ns;
  P.ng = ng;
  P.K = K;
  P.batch = batch;
  P.npad = tr_npad(ns);
  P.kind_bf16 = precision == TNQ_PREC_BF16X3 ? 1 : 0;
  P.split = precision == TNQ_PREC_TF32 ? 0 : 1;
  const int k_step = P.kind_bf16 ? 8 : 4;  // complex values per 32-byte MMA K step
  P.nks = (K + k_step - 1) / k_step;
  P.atoms = tr_atoms(K, P.kind_bf16 != 0);
  const size_t bp_all = tr_bprime_bytes(ns, K, batch, P.kind_bf16 != 0);
  const TrStages ts = K > TR_RESIDENT_KMAX ? tr_stages_streamed(P.atoms, P.npad) : tr_stages(P.atoms, bp_all);
  if (ts.stages < 2) return cudaErrorNotSupported;
  P.stream_bp = ts.stream ? 1 : 0;
  P.bp_part = uint32_t(ts.patoms) * uint32_t(P.npad) * TR_ROW_BYTES;
  P.bp_glob = reinterpret_cast<const uint8_t*>(scratch);
  if (P.stream_bp && (!scratch || scratch_bytes < bp_all || (reinterpret_cast<uintptr_t>(scratch) & 255)))
    return cudaErrorNotSupported;
  P.kparts = ts.kparts;
  P.patoms = ts.patoms;
  P.stages = ts.stages;
  P.nks_part = P.kparts == 1 ? P.nks : 4 * P.patoms;  // parts of several atoms hold whole atoms of K
  P.kc = P.kparts == 1 ? K : P.patoms * TR_ROW_BYTES / (2 * (P.kind_bf16 ? 2 : 4));
  P.nacc = P.npad <= 64 ? 4 : 2;  // TMEM: acc_cols * nacc <= 512 columns
  // The split modes keep the correction products in a second TMEM buffer
  // beside the hi*hi one, so that hi*hi and hi*lo come from one MMA of
  // N = 2 npad over S' hi and lo rows (two MMAs per K step instead of three;
  // each MMA instruction has a fixed issue cost of the order of 10^2 cycles,
  // which dominates these short-K tiles) and the TF32 sums escape most of the
  // truncating accumulation (the corrections, about 2^-9 of the sum, are added
  // once in the epilogue).  N = 2 npad <= 256 bounds it to npad <= 128.
  P.dual = (P.split && P.npad <= 128) ? 1 : 0;
  P.merged = P.dual;
  P.acc_cols = P.npad * (P.dual ? 2 : 1);
  // Two CTAs per SM where a launch fits in half an SM: at least two stages
  // beside S' in TR_SMEM_HALF bytes and two TMEM buffers in 256 columns.
  // Measured on pair contractions: BF16x3 16 x 2^24 x 16 3.6 -> 4.5 TB/s,
  // TF32x3 8 x 2^23 x 8 2.7 -> 3.4; TF32x3 16 x 2^24 x 16 unchanged (its
  // hi/lo split arithmetic, not the warp count, bounds it there).
  bool two = false;
  if (!P.stream_bp && 2 * P.acc_cols <= 256) {
    const size_t stage_bytes = size_t(2) * TR_ATOM_BYTES * P.patoms;
    int st2 = P.stages;
    while (st2 > 2 && size_t(st2) * stage_bytes + bp_all + 1024 > size_t(TR_SMEM_HALF)) --st2;
    if (size_t(st2) * stage_bytes + bp_all + 1024 <= size_t(TR_SMEM_HALF)) {
      two = true;
      P.stages = st2;
      P.nacc = std::min(P.nacc, 256 / P.acc_cols);
    }
  }
  const int ch = (two || P.kc <= 8) ? 8 : 16;
  P.nchunks = (P.kc + ch - 1) / ch;
  P.pairs = gd.nk >= 1 && gd.kpos[0] == 0;
  P.row_tab = gd.nrow - 7 <= 4 * TR_ROWTAB_DIGITS ? 1 : 0;
  for (int j = 7; j < gd.nrow; ++j)
    if (gd.rowpos[j] >= 32) P.row_tab = 0;
  P.s_stride = s_stride_out;
  P.g_stride = g_stride_out;
  P.tiles_per_h = ng / 128;
  P.total_tiles = (long long)P.tiles_per_h * batch;
  // 32-bit tile counters: cursors run up to 2 items (4 grid strides) past the end
  if (P.total_tiles + 8ll * std::max(1, sm_count) > 0xffffffffll) return cudaErrorNotSupported;
  P.slice_id = slice_id;
  // instruction descriptor: FP32 accumulator, A/B format (TF32 = 2, BF16 = 1), K-major, N >> 3, M >> 4
  const uint32_t fmt = P.kind_bf16 ? 1u : 2u;
  P.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(P.npad >> 3) << 17) | (uint32_t(128 >> 4) << 24);
  P.idesc2 = (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t((2 * P.npad) >> 3) << 17) | (uint32_t(128 >> 4) << 24);
  P.C = reinterpret_cast<float2*>(C);
  P.acc = reinterpret_cast<double2*>(acc);
  P.err = err;
  const long long grid = std::min<long long>(P.total_tiles, (two ? 2 : 1) * std::max(1, sm_count));
  const size_t smem = size_t(P.stages) * (2 * P.patoms * TR_ATOM_BYTES + (P.stream_bp ? 2 * size_t(P.bp_part) : 0)) +
                      (P.stream_bp ? 0 : bp_all) + 1024;
  if (P.stream_bp) {
    // S' of every batch entry, expanded once into the scratch for this launch
    const long long n = (long long)batch * P.npad * P.nks * (32 / (P.kind_bf16 ? 2 : 4));
    const unsigned blocks = unsigned(std::min<long long>((n + 255) / 256, 1024));
    build_bprime_kernel<<<blocks, 256, 0, st>>>(P, reinterpret_cast<uint8_t*>(scratch));
  }
  const int mode = P.kind_bf16 ? 2 : (P.split ? 1 : 0);
  const TrKernel k = two ? kTrKernels2[mode] : kTrKernels[ch == 16 ? 1 : 0][mode];
  k<<<unsigned(grid), TR_THREADS, smem, st>>>(P);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cgemm_tc_rows(const void* Ssmall, const void* Gsrc, const GatherDesc& gd, void* C, void* acc, int ns,
                                 int ng, int K, int batch, long long s_stride_out, long long g_stride_out, int slice_id,
                                 int precision, int* err, int sm_count, cudaStream_t st, void* scratch,
                                 size_t scratch_bytes) {
  if (!tc_rows_supported(ns, ng, K, batch, gd.nrow, precision) || !err) return cudaErrorNotSupported;
  if (gd.nk > 8 || gd.nrow > 32 || (1 << gd.nk) != K) return cudaErrorInvalidValue;
  cudaError_t pe = tc_rows_prepare();
  if (pe != cudaSuccess) return pe;
  const bool bf16 = precision == TNQ_PREC_BF16X3;
  if (K > TR_RESIDENT_KMAX)
    return launch_tc_rows_one(Ssmall, Gsrc, gd, C, acc, ns, ng, K, batch, s_stride_out, g_stride_out, slice_id,
                              precision, err, sm_count, st, scratch, scratch_bytes);
  const size_t bp_all = tr_bprime_bytes(ns, K, batch, bf16);
  if (bp_all <= size_t(TR_BPRIME_BUDGET) && tr_stages(tr_atoms(K, bf16), bp_all).stages >= 2)
    return launch_tc_rows_one(Ssmall, Gsrc, gd, C, acc, ns, ng, K, batch, s_stride_out, g_stride_out, slice_id,
                              precision, err, sm_count, st);
  // S' of every batch entry does not fit: one launch per entry, whose batch
  // bits (the row bits above the ng bits) become extra slice bits of G
  int gbits = 0;
  while ((1 << gbits) < ng) ++gbits;
  const int hbits = gd.nrow - gbits;
  if (hbits < 0 || (1 << hbits) != batch || gd.n_slice + hbits > 30) return cudaErrorNotSupported;
  GatherDesc g1 = gd;
  g1.nrow = gbits;
  for (int j = 0; j < hbits; ++j) g1.slice_src[gd.n_slice + j] = gd.rowpos[gbits + j];
  g1.n_slice = gd.n_slice + hbits;
  const float2* S = reinterpret_cast<const float2*>(Ssmall);
  for (int h = 0; h < batch; ++h) {
    const size_t ob = size_t(h) * ns * ng;
    cudaError_t e = launch_tc_rows_one(S + size_t(h) * ns * K, Gsrc, g1,
                                       C ? static_cast<void*>(reinterpret_cast<float2*>(C) + ob) : nullptr,
                                       acc ? static_cast<void*>(reinterpret_cast<double2*>(acc) + ob) : nullptr, ns,
                                       ng, K, 1, s_stride_out, g_stride_out, slice_id | (h << gd.n_slice), precision,
                                       err, sm_count, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace tnq
