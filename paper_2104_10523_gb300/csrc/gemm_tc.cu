// Placeholder until the tcgen05 kernel lands: reports the shape as unsupported.
#include "gemm_tc.cuh"

namespace tnq {

cudaError_t launch_cgemm_tc(const TcGemmArgs&, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace tnq
