// k_backward.cu -- adjoint of the rasterizer (placeholder until written).
#include "gs_internal.cuh"

namespace gs {

cudaError_t launch_backward(const gs_plan *, void *, const float *, const float *,
                            const int32_t *, const float *, float *, float *, float *, float *,
                            float *, float *, float *, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace gs
