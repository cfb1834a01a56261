// Device kernels and their launch descriptors (shared by the executor and the
// pairwise-contraction entry point).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tnq {

// Operand formats written by the permute kernel.
enum PermMode {
  PM_C64 = 0,          // complex64 copy in the new order
  PM_AEXP_F32 = 1,     // A' = [[re,-im],[im,re]] real expansion, FP32 (2 rows x 2K floats per complex row)
  PM_AEXP_TF32 = 2,    // as above, rounded to TF32
  PM_AEXP_TF32X3 = 3,  // as above, hi/lo TF32 split into dst0/dst1
  PM_AEXP_BF16X3 = 4,  // as above, hi/lo BF16 split
  PM_B_TF32 = 5,       // complex64 rounded to TF32
  PM_B_TF32X3 = 6,     // complex64 hi/lo TF32 split
  PM_B_BF16X3 = 7      // complex pairs as bf16x2, hi/lo split
};

struct PermDesc {
  int r;                       // destination rank
  int u;                       // bits staged per tile
  int n_outer;                 // r - u
  int kbits;                   // A' expansion: number of K bits (lowest destination bits)
  int mode;
  int n_slice;                 // slice-id bits
  int tile_src[16];            // i-th tile bit (source order): its source bit position
  int tile_dst_sorted[16];     // tile bits in destination order: destination bit position
  int tile_srcidx_of_dst[16];  // j-th tile bit in destination order -> its source-order index
  int outer_src[32];
  int outer_dst[32];
  int slice_src[32];           // source bit of slice bit j, or -1
};

void build_perm_desc(const int* src_labels, int src_rank, const int* dst_labels, int dst_rank,
                     const int* slice_labels, int n_slice, int mode, int kbits, PermDesc* d);

cudaError_t launch_permute(const PermDesc& d, const void* src, void* dst0, void* dst1, int slice_id,
                           int sm_count, cudaStream_t st);

// C[h][m][n] = sum_k A[h][m][k] * B[h][n][k] (complex64, FP32 FFMA); with acc
// non-null the result is added in FP64 to acc (same layout) instead of stored.
// With splits > 1 the K range is cut into `splits` parts whose FP32 partial
// products go to part[s][h][m][n]; launch_reduce_splits then forms C or acc.
cudaError_t launch_cgemm_simt(const void* A, const void* B, void* C, void* acc, void* part, int splits, int M,
                              int N, int K, int batch, cudaStream_t st);
cudaError_t launch_reduce_splits(const void* part, int splits, size_t n, void* C, void* acc, int sm_count,
                                 cudaStream_t st);

// Skinny steps (see skinny.cu).  rows: C = S x G^T for a small operand S of
// ns <= 32 rows; output element (h, s, g) at h*ns*ng + s*s_stride + g*g_stride.
// dot: M, N <= 8; always writes FP32 partials [splits][batch][M][N].
cudaError_t launch_cgemm_rows(const void* Ssmall, const void* Gbig, void* C, void* acc, void* part, int splits,
                              int ns, int ng, int K, int batch, long long s_stride_out, long long g_stride_out,
                              cudaStream_t st);
cudaError_t launch_cdot(const void* A, const void* B, void* part, int splits, int M, int N, int K, int batch,
                        cudaStream_t st);
// Operand of the dot kernel addressed through bit deposits: element (row r of
// batch entry h, k) sits at p + dep(h * rows + r, rowpos) + dep(k, kpos), with
// kmask = OR of 1 << kpos[j].  kpos[0] must be 0 (16-byte pair loads) and
// kpos must increase.
struct DotOp {
  const float2* p;              // slice offset already added
  unsigned long long kmask;
  int nk, nrow;
  signed char kpos[40];
  signed char rowpos[24];
};
DotOp dot_contiguous(const void* p, int rows, int K, int batch);
cudaError_t launch_cdot_ops(const DotOp& A, const DotOp& B, void* part, int splits, int M, int N, int K, int batch,
                            cudaStream_t st);

// Bit positions (in the large operand's stored layout) of its row index (the
// N or M bits, then the batch bits) and of its K bits, plus sliced labels.
struct GatherDesc {
  int nrow;
  int rowpos[32];
  int nk;
  int kpos[8];
  int n_slice;
  int slice_src[32];
};
// rows kernel with K <= 32 reading the large operand in place (fused permute).
cudaError_t launch_cgemm_rows_gather(const void* Ssmall, const void* Gsrc, const GatherDesc& gd, void* C, void* acc,
                                     int ns, int ng, int K, int batch, long long s_stride_out, long long g_stride_out,
                                     int slice_id, cudaStream_t st);

// Projection leaves j < n_proj at leaves_base + j * stride_bytes:
// P_j[(b << 1) | x] = [bits[b * row_len + tab[j]] == x] for b < n_valid, else 0.
// tab (device) also lists, after the n_proj entries, the n_open row entries
// that must hold -1 (open qubits).  Entries of another value set *err_flag.
cudaError_t launch_proj_fill(void* leaves_base, size_t stride_bytes, int n_proj, int n_open, const int* tab,
                             int row_len, int batch_log2, const int8_t* bits, int64_t n_valid, int* err_flag,
                             cudaStream_t st);

// out[b * 2^n_open + o] = acc[root_index(b, o)] for b < n_valid (complex128;
// only the real part, as one double, when real_only), where root_index =
// sum_j bit_j(b) << pos[j] + sum_i bit_(n_open-1-i)(o) << open_pos[i].
cudaError_t launch_finalize(const void* acc, void* out, int64_t n_valid, const int* pos_table, int n_pos,
                            const int* open_pos, int n_open, bool real_only, cudaStream_t st);

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st);

}  // namespace tnq
