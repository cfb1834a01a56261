// GPU executor of a plan: per batch of bitstrings (and trajectories) it runs
// every slice's pairwise contraction sequence and sums the slices in FP64.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace tnq {

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = TNQ_PREC_FP32;
  int sm_count = 0;
};

tnq_status exec_bind(Ctx* ctx, Plan* p, void* ws, size_t bytes);
tnq_status exec_amplitudes(Ctx* ctx, Plan* p, int64_t n_bs, const int8_t* bits, double* out);
tnq_status exec_noisy(Ctx* ctx, Plan* p, int64_t n_traj, uint64_t seed, int64_t n_bs, const int8_t* bits,
                      double* p_out, double* se_out);
tnq_status exec_contract_pair(Ctx* ctx, const void* A, int ra, const int* al, const void* B, int rb,
                              const int* bl, void* C, int rc, const int* cl, void* ws, size_t ws_bytes);
size_t contract_workspace_bytes(int precision, int ra, int rb, int rc);

tnq_status cuda_fail(cudaError_t e, const char* what);

}  // namespace tnq

struct tnq_ctx { tnq::Ctx c; };
