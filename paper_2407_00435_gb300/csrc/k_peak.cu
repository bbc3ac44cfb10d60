// k_peak.cu -- issue-rate probe of the FP32 FMA pipe and the special-function
// unit (ex2), the two units the rasterizer's inner loop is bound by.  Every
// thread runs 8 independent dependency chains so that the pipes, not the
// latency of one chain, limit the rate.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_internal.cuh"
#include "raster.cuh"

namespace gs {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_peak(int iters, float seed, float *sink) {
  float x[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) x[c] = seed * (float)(threadIdx.x + c + 1) * 1e-3f;
  const float b = 0.9999f, d = 1e-4f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) {
      if (KIND == 0) x[c] = fmaf(x[c], b, d);                 // converges to 1: no denormals
      else x[c] = ex2_approx(-x[c]);                          // stays in [0.5, 1]
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += x[c];
  if (s == 12345.678f) *sink = s;   // practically never taken; keeps the chains alive
}

}  // namespace gs

extern "C" gs_status gs_peak_probe(int32_t kind, int32_t iters, float *d_sink, int64_t *ops,
                                   cudaStream_t stream) {
  using namespace gs;
  if ((kind != 0 && kind != 1) || iters < 1 || !d_sink || !ops) return GS_ERR_INVALID_ARG;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GS_ERR_CUDA;
  cudaError_t e = kind == 0
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_peak<0>, kPeakThreads, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_peak<1>, kPeakThreads, 0);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  const int grid = sms * (per > 0 ? per : 1);
  if (kind == 0) k_peak<0><<<grid, kPeakThreads, 0, stream>>>(iters, 1.0f, d_sink);
  else k_peak<1><<<grid, kPeakThreads, 0, stream>>>(iters, 1.0f, d_sink);
  if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
  *ops = (int64_t)grid * kPeakThreads * (int64_t)iters * kPeakChains;
  return GS_OK;
}
