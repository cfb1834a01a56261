// Pairwise contraction that allocates no device memory.
//
// Some callers cannot allocate device memory while they run: programs that
// hand all device memory to their own pool allocator up front and forbid any
// other allocation, and latency-critical loops that cannot afford the device
// synchronisation cudaFree implies.  For them this entry point runs the same
// permute + GEMM contraction as tnq_contract_pair, but its scratch (converted
// operands, split-K partials, the error flag) lives in one file-scope device
// array of fixed size that is part of the loaded library.
//
// Facts a caller must know:
//   * the array (kNoAllocScratchBytes) is device memory of the library's
//     module on each GPU; with CUDA's lazy module loading (the default) the
//     module, and so the array, is committed on a device when the first call
//     there looks the array up, and it stays until the process exits.  A
//     caller whose own pool takes all device memory must make that first call
//     before the pool reserves it;
//   * the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress with that device current) and caches it; make that
//     first call before any stream capture;
//   * a call returns after its contraction has completed (it reads the error
//     flag back and synchronizes the context's stream);
//   * the context's per-kernel timing records (tnq_ctx_set_timing) are not
//     taken for these calls;
//   * all calls share the array and it keeps the last call's contents: calls
//     that overlap on the GPU (different streams, threads or contexts without
//     ordering between them) race on it and give wrong results;
//   * only what must start at zero (the error flag) is cleared per call; every
//     other scratch byte is written before it is read;
//   * a contraction needing more scratch than the array holds is rejected with
//     TNQ_ERR_INVALID_ARG and a message naming both sizes.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "executor.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

// In host code this name is a host-side stand-in, not a device address: only
// the pointer cudaGetSymbolAddress returns may be handed to a kernel.
static __device__ __align__(256) unsigned char tnq_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};

}  // namespace

extern "C" tnq_status tnq_contract_pair_noalloc(tnq_ctx* c, const void* A, int ra, const int* a_labels,
                                                const void* B, int rb, const int* b_labels, void* C, int rc,
                                                const int* c_labels) {
  using namespace tnq;
  if (!c || !A || !B || !C) return fail(TNQ_ERR_INVALID_ARG, "NULL argument");
  if ((ra && !a_labels) || (rb && !b_labels) || (rc && !c_labels))
    return fail(TNQ_ERR_INVALID_ARG, "NULL label array");
  if (ra < 0 || rb < 0 || rc < 0 || ra > 31 || rb > 31 || rc > 31)
    return fail(TNQ_ERR_INVALID_ARG, "ranks must be in [0, 31]");
  const Ctx& user = c->c;
  if (user.device < 0 || user.device >= kMaxDevices) return fail(TNQ_ERR_INVALID_ARG, "device ordinal too large");
  const size_t need = contract_workspace_bytes(user.precision, ra, rb, rc);
  if (need > kNoAllocScratchBytes)
    return fail(TNQ_ERR_INVALID_ARG, "contraction needs " + std::to_string(need) +
                                         " bytes of scratch, more than the " +
                                         std::to_string(kNoAllocScratchBytes) +
                                         " bytes of the static scratch of tnq_contract_pair_noalloc");
  cudaError_t e = cudaSetDevice(user.device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[user.device]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, tnq_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(tnq_noalloc_scratch)");
      g_scratch[user.device] = p;
    }
    scratch = g_scratch[user.device];
  }
  // A context copy without the timing recorder (which would create events).
  Ctx run;
  run.device = user.device;
  run.stream = user.stream;
  run.precision = user.precision;
  run.sm_count = user.sm_count;
  run.tc_min_work = user.tc_min_work;
  tnq_status st = exec_contract_pair(&run, A, ra, a_labels, B, rb, b_labels, C, rc, c_labels, scratch,
                                     kNoAllocScratchBytes);
  c->c.launches += run.launches;
  return st;
}
