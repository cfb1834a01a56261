// Complex GEMM on the tcgen05 tensor cores (TMEM accumulators, TMA-staged
// operands).  C[h][m][n] = sum_k A[h][m][k] B[h][n][k] computed as the real
// product of the expansion A' (2M x 2K, rows (m,re|im), columns (k,re|im)) with
// B (N rows of K interleaved complex values), FP32 accumulation.
#pragma once

#include <cuda_runtime.h>

namespace tnq {

struct TcGemmArgs {
  const void* a_hi = nullptr;  // A' (fp32 / tf32 / bf16 hi part), [batch][2M][2K]
  const void* a_lo = nullptr;  // lo part (split modes) or null
  const void* b_hi = nullptr;  // B, [batch][N][2K] reals
  const void* b_lo = nullptr;
  void* c = nullptr;           // complex64 [batch][M][N], or
  void* acc = nullptr;         // complex128 accumulator (added to) when non-null
  int M = 0, N = 0, K = 0, batch = 1;
  int precision = 0;           // tnq_precision
  int* err = nullptr;          // device flag, set when a bounded wait runs out
  int splits = 1;              // requested K splits (partials to `part`, reduced by the caller)
  void* part = nullptr;        // FP32 partials [splits][batch][M][N] complex
  int* splits_used = nullptr;  // out: splits actually launched
};

// One-time set-up (driver entry point, shared-memory limit); call outside capture.
cudaError_t tc_gemm_prepare();

// Whether a GEMM of this shape and precision runs on the tensor cores.
bool tc_gemm_supported(int M, int N, int K, int precision);

// Returns cudaErrorNotSupported when the shape cannot run on the tensor cores.
cudaError_t launch_cgemm_tc(const TcGemmArgs& g, int sm_count, cudaStream_t st);

struct GatherDesc;

// Tall-skinny tensor-core GEMM (gemm_tc_rows.cu): out[h][s][g] (strides
// s_stride_out, g_stride_out; batch stride ns * ng) = sum_k S[h][s][k] G[h][g][k]
// for a small operand S ([batch][ns][K] complex64, ns <= 128, K <= 256) and a
// large one G read in
// its stored bit order through gd, split into BF16 or TF32 hi/lo parts in
// shared memory.  Adds into the FP64 acc when non-null, else writes C.
// K up to 64 keeps S' whole in shared memory; K of 128 or 256 streams it per
// K-part from a global copy built in `scratch` (tc_rows_scratch_bytes, 256-byte
// aligned; cudaErrorNotSupported when it is missing or too small).
bool tc_rows_supported(int ns, int ng, int K, int batch, int nrow, int precision);
size_t tc_rows_scratch_bytes(int ns, int K, int batch, int precision);
cudaError_t tc_rows_prepare();
cudaError_t launch_cgemm_tc_rows(const void* Ssmall, const void* Gsrc, const GatherDesc& gd, void* C, void* acc, int ns,
                                 int ng, int K, int batch, long long s_stride_out, long long g_stride_out, int slice_id,
                                 int precision, int* err, int sm_count, cudaStream_t st, void* scratch = nullptr,
                                 size_t scratch_bytes = 0);

}  // namespace tnq
