// Internal interface between the step kernels and the learned-guess MLP (mlp.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/grte.h"

namespace grte {
// y[i] = network(feat[6*i .. 6*i+5]) for i < n (un-standardised), on `stream`.
cudaError_t mlp_guess_launch(grte_mlp_t mlp, const float* feat, int64_t n, float* y, cudaStream_t stream);
}  // namespace grte
