// Kraus-trajectory leaf builder (stochastic noise via Kraus operators).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tnq {}  // namespace tnq
