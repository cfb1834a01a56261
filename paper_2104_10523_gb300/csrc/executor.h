// GPU executor of a plan: per batch of bitstrings (and trajectories) it runs
// every slice's pairwise contraction sequence and sums the slices in FP64.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace tnq {

// One kernel launch as seen by the optional timing recorder.
struct KernelRecord {
  int kind;        // 0 permute, 1 SIMT GEMM, 2 tensor-core GEMM, 3 other, 4 skinny (rows/dot) GEMM,
                   // 5 tall-skinny tensor-core GEMM
  int step;        // plan step index (-1 outside a plan)
  int nH, nM, nN, nK;
  double flops;    // algorithmic flops (8 per complex multiply-add)
  double bytes;    // algorithmic bytes moved
  float ms;        // CUDA-event duration on the launching stream
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = TNQ_PREC_FP32;
  int sm_count = 0;
  double tc_min_work = 1 << 18;  // complex MACs below which a step stays on the CUDA cores
  uint64_t launches = 0;         // kernels launched by this context (cumulative)
  bool timing = false;           // record CUDA events around every kernel
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, KernelRecord>> pending;  // (event index, record)
  std::vector<KernelRecord> records;
  int cur_step = -1;
  int kernel_policy = 0;         // TNQ_KERNELS_DEFAULT or TNQ_KERNELS_TENSOR_CORES
  bool use_graphs = true;        // replay full batches from a captured CUDA graph
  cudaStream_t capture_stream = nullptr;  // private stream graphs are captured on
};

void plan_release_graph(Plan* p);
tnq_status exec_autotune(Ctx* ctx, Plan* p, int reps, int* n_tc, int* n_cuda);

// Timing helpers: bracket a launch when ctx->timing is set.
int timing_begin(Ctx* ctx);
void timing_end(Ctx* ctx, int slot, const KernelRecord& r);
tnq_status timing_collect(Ctx* ctx);  // after a stream sync

tnq_status exec_bind(Ctx* ctx, Plan* p, void* ws, size_t bytes);
tnq_status exec_amplitudes(Ctx* ctx, Plan* p, int64_t n_bs, const int8_t* bits, double* out);
tnq_status exec_amplitudes_range(Ctx* ctx, Plan* p, int64_t n_bs, const int8_t* bits, int64_t slice_begin,
                                 int64_t slice_count, double* out);
tnq_status exec_noisy(Ctx* ctx, Plan* p, int64_t n_traj, uint64_t seed, int64_t n_bs, const int8_t* bits,
                      double* p_out, double* se_out);
tnq_status exec_traj_amplitudes(Ctx* ctx, Plan* p, uint64_t seed, int64_t traj_begin, int64_t n_traj, int64_t n_bs,
                                const int8_t* bits, double* out);
tnq_status exec_expectation(Ctx* ctx, Plan* p, const double* coeffs, double* value, double* term_values);
tnq_status exec_contract_pair(Ctx* ctx, const void* A, int ra, const int* al, const void* B, int rb,
                              const int* bl, void* C, int rc, const int* cl, void* ws, size_t ws_bytes);
size_t contract_workspace_bytes(int precision, int ra, int rb, int rc);

tnq_status cuda_fail(cudaError_t e, const char* what);

}  // namespace tnq

struct tnq_ctx { tnq::Ctx c; };
