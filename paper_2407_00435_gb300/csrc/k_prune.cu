// k_prune.cu -- efficiency-aware pruning and scale decay (Sec. 3.2-3.4):
// the computational efficiency of each point from a render's statistics,
// its maximum over poses, the mask of the lowest-efficiency fraction, stable
// compaction of the scene, and the weighted-scale loss with its gradient.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_internal.cuh"

namespace gs {

// CE_i = Val_i / Comp_i (Eq. 2) with Val = pixels dominated (stats row 3) and
// Comp = tiles whose list holds the point (row 0); max over poses.
__global__ void k_ce_update(long long n, const uint32_t *stats, float *ce_max) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint32_t comp = stats[i], val = stats[3 * n + i];
    if (comp == 0u) continue;
    const float ce = __fdiv_rn((float)val, (float)comp);
    ce_max[i] = fmaxf(ce_max[i], ce);
  }
}

// keep[i] = 0 for the k points ranked first by (CE, index).
__global__ void k_mark_pruned(long long n, long long k, const uint32_t *order, uint8_t *keep) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x)
    keep[order[r]] = r < k ? 0u : 1u;
}

// ---- stable compaction by a keep mask (reduce-then-scan over block ranges)
struct CompactArgs {
  long long n;
  int S3;                        // SH floats per point
  const uint8_t *keep;
  const float *means, *scales, *quats, *opac, *sh;
  float *o_means, *o_scales, *o_quats, *o_opac, *o_sh;
  unsigned long long *bsum;      // [G] per-block kept counts -> bases
  int blocks;
  unsigned long long *n_out;
};

__device__ __forceinline__ void compact_range(const CompactArgs &a, int b, long long &i0,
                                              long long &i1) {
  const long long q = (a.n + a.blocks - 1) / a.blocks;
  i0 = (long long)b * q < a.n ? (long long)b * q : a.n;
  i1 = i0 + q < a.n ? i0 + q : a.n;
}

__global__ void __launch_bounds__(256) k_keep_count(CompactArgs a) {
  __shared__ unsigned long long s_w[8];
  long long i0, i1;
  compact_range(a, blockIdx.x, i0, i1);
  unsigned long long c = 0;
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) c += a.keep[i] ? 1u : 0u;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    a.bsum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_keep_scan(CompactArgs a) {
  __shared__ unsigned long long s_w[32];
  const int G = a.blocks, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int per = (G + 1023) / 1024;
  const int r0 = threadIdx.x * per < G ? threadIdx.x * per : G;
  const int r1 = r0 + per < G ? r0 + per : G;
  unsigned long long local = 0;
  for (int r = r0; r < r1; ++r) local += a.bsum[r];
  unsigned long long incl = local;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  unsigned long long woff = 0, total = 0;
  for (int w = 0; w < 32; ++w) {
    if (w < warp) woff += s_w[w];
    total += s_w[w];
  }
  unsigned long long run = woff + incl - local;
  for (int r = r0; r < r1; ++r) {
    const unsigned long long c = a.bsum[r];
    a.bsum[r] = run;
    run += c;
  }
  if (threadIdx.x == 0) *a.n_out = total;
}

// Each block copies its range's kept points in order (a warp-wide ballot
// prefix gives each kept point its place).
__global__ void __launch_bounds__(256) k_keep_scatter(CompactArgs a) {
  __shared__ unsigned long long s_w[8];
  __shared__ unsigned long long s_carry;
  long long i0, i1;
  compact_range(a, blockIdx.x, i0, i1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = a.bsum[blockIdx.x];
  __syncthreads();
  for (long long base = i0; base < i1; base += blockDim.x) {
    const long long i = base + threadIdx.x;
    const bool k = i < i1 && a.keep[i];
    const uint32_t bal = __ballot_sync(0xffffffffu, k);
    if (lane == 0) s_w[warp] = __popc(bal);
    __syncthreads();
    unsigned long long woff = 0, tot = 0;
    for (int w = 0; w < 8; ++w) {
      if (w < warp) woff += s_w[w];
      tot += s_w[w];
    }
    if (k) {
      const long long o = (long long)(s_carry + woff + __popc(bal & ((1u << lane) - 1u)));
      for (int c = 0; c < 3; ++c) {
        a.o_means[3 * o + c] = a.means[3 * i + c];
        a.o_scales[3 * o + c] = a.scales[3 * i + c];
      }
      for (int c = 0; c < 4; ++c) a.o_quats[4 * o + c] = a.quats[4 * i + c];
      a.o_opac[o] = a.opac[i];
      for (int c = 0; c < a.S3; ++c) a.o_sh[(long long)a.S3 * o + c] = a.sh[(long long)a.S3 * i + c];
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry += tot;
    __syncthreads();
  }
}

// WS = (1/N) sum_i S_i G_i (Eq. 3), G_i = (U_i > T)(U_i - T) (Eq. 4), S_i the
// largest of the point's scales, U_i = tiles that blended it (stats row 1).
// Adds gamma dWS/ds to d_scales (first largest axis) when given.
__global__ void __launch_bounds__(256) k_weighted_scale(long long n, const float *scales,
                                                        const uint32_t *stats, float T,
                                                        float gamma, double *ws_out,
                                                        float *d_scales) {
  __shared__ double s_w[8];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float u = (float)stats[n + i];
    const float G = u > T ? u - T : 0.0f;
    if (G == 0.0f) continue;
    const float s0 = scales[3 * i], s1 = scales[3 * i + 1], s2 = scales[3 * i + 2];
    int k = 0;
    float S = s0;
    if (s1 > S) { S = s1; k = 1; }
    if (s2 > S) { S = s2; k = 2; }
    acc += (double)S * (double)G;
    if (d_scales) d_scales[3 * i + k] += gamma * G / (float)n;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    if (t != 0.0) atomicAdd(ws_out, t / (double)n);
  }
}

}  // namespace gs

using namespace gs;

namespace {
unsigned grid_for(long long n, int threads, int cap) {
  const long long b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}
}  // namespace

extern "C" {

gs_status gs_ce_update(int64_t n, const uint32_t *stats, float *ce_max, cudaStream_t stream) {
  if (n < 0 || (n > 0 && (!stats || !ce_max))) return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  k_ce_update<<<grid_for(n, 256, 4096), 256, 0, stream>>>(n, stats, ce_max);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_prune_mask(gs_plan *p, void *ws, int64_t n, const float *ce_max, double fraction,
                        uint8_t *keep, cudaStream_t stream) {
  if (!p || !ws || n < 0 || (n > 0 && (!ce_max || !keep))) return GS_ERR_INVALID_ARG;
  if (!(fraction >= 0.0 && fraction <= 1.0)) return GS_ERR_INVALID_ARG;
  if (n > p->max_visible) return GS_ERR_INVALID_ARG;   // the sort buffers hold max_visible keys
  if (n == 0) return GS_OK;
  const long long k = (long long)(fraction * (double)n);   // floor for non-negative values
  cudaError_t e = launch_sort_indices(p, ws, reinterpret_cast<const uint32_t *>(ce_max), n, stream);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  k_mark_pruned<<<grid_for(n, 256, 4096), 256, 0, stream>>>(n, k, region<uint32_t>(p, ws, R_DVAL_A),
                                                           keep);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_compact_points(gs_plan *p, void *ws, int64_t n, int32_t sh_degree, const uint8_t *keep,
                            const gs_scene *in, gs_scene *out, uint64_t *n_out,
                            cudaStream_t stream) {
  if (!p || !ws || !keep || !in || !out || !n_out || n < 0) return GS_ERR_INVALID_ARG;
  if (sh_degree < 0 || sh_degree > 3) return GS_ERR_INVALID_ARG;
  if (n > 0 && (!in->means || !in->scales || !in->quats || !in->opacities || !in->sh ||
                !out->means || !out->scales || !out->quats || !out->opacities || !out->sh))
    return GS_ERR_INVALID_ARG;
  CompactArgs a = {};
  a.n = n;
  a.S3 = 3 * (sh_degree + 1) * (sh_degree + 1);
  a.keep = keep;
  a.means = in->means; a.scales = in->scales; a.quats = in->quats; a.opac = in->opacities;
  a.sh = in->sh;
  a.o_means = const_cast<float *>(out->means); a.o_scales = const_cast<float *>(out->scales);
  a.o_quats = const_cast<float *>(out->quats); a.o_opac = const_cast<float *>(out->opacities);
  a.o_sh = const_cast<float *>(out->sh);
  // the u64 half of the sort's block table serves as scratch
  a.bsum = reinterpret_cast<unsigned long long *>(region<uint32_t>(p, ws, R_BSUM) +
                                                  (size_t)p->sort_blocks * kSortSub * 256);
  a.blocks = p->sort_blocks;
  a.n_out = reinterpret_cast<unsigned long long *>(n_out);
  if (n == 0) {
    return cudaMemsetAsync(n_out, 0, sizeof(uint64_t), stream) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
  }
  k_keep_count<<<a.blocks, 256, 0, stream>>>(a);
  k_keep_scan<<<1, 1024, 0, stream>>>(a);
  k_keep_scatter<<<a.blocks, 256, 0, stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_weighted_scale(int64_t n, const float *scales, const uint32_t *stats, float T,
                            float gamma, double *ws_out, float *d_scales, cudaStream_t stream) {
  if (n < 0 || !ws_out || (n > 0 && (!scales || !stats))) return GS_ERR_INVALID_ARG;
  if (cudaMemsetAsync(ws_out, 0, sizeof(double), stream) != cudaSuccess) return GS_ERR_CUDA;
  if (n == 0) return GS_OK;
  k_weighted_scale<<<grid_for(n, 256, 2048), 256, 0, stream>>>(n, scales, stats, T, gamma, ws_out,
                                                              d_scales);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // extern "C"
