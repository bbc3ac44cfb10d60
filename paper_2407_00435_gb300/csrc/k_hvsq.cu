// k_hvsq.cu -- the eccentricity-aware visual quality metric HVSQ (Sec. 2.2,
// the HVSQ equation) and its gradient, used per quality region as the
// quality loss of level training (Sec. 4.3).
//
// For pixel i of an altered image a and a reference r, with P_i the square
// box of half-width r_i around i (clipped to the image):
//   term_i = sum_c (mean_c(a, P_i) - mean_c(r, P_i))^2
//                + (std_c(a, P_i) - std_c(r, P_i))^2
// and the HVSQ of a region is the mean of term_i over its pixels.  r_i grows
// with the pixel's eccentricity: r_base + #{j : |p_i - g| >= f tan theta_j}
// (thresholds given by the caller); regions are the foveation levels
// 1 + #{k : |p_i - g| >= f tan ring_k}.  Both integer decisions are taken
// in FP32 with the expressions of the renderer's ring test.
//
// Data path (all FP64 where sums are formed):
//   rows     per pixel and channel, v = x - 1/2 and v^2 of both images,
//            prefix-summed along the image row into 12 planes of
//            (H+1) x (W+1) (first row and column zero)
//   columns  prefix sums down the columns: summed-area tables, so that a
//            box sum is 4 lookups (shifting by 1/2 keeps the tables small)
//   stats    per pixel: box statistics, the term, its region's sum; for the
//            gradient the pooling's coefficients A, B (d L / d x_q =
//            sum over poolings containing q of A + (x_q - 1/2) B) are added
//            at the 4 corners of its box in 6 difference planes
//   scan     2D prefix of the difference planes: at q, the sum of A and B
//            over every box that contains q
//   grad     d_alt = A + (a - 1/2) B
// Scratch: 18 FP64 planes of (H+1)(W+1) plus region accumulators.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kMaxPool = 64;
constexpr int kMaxRings = GS_MAX_LEVELS - 1;
constexpr int kValPlanes = 12;   // per channel: a - 1/2, (a - 1/2)^2, r - 1/2, (r - 1/2)^2
constexpr int kDiffPlanes = 6;   // per channel: A, B

struct HvsqArgs {
  const float *alt, *ref;
  int W, H;
  float gx, gy, focal;
  int n_rings, n_pool, r_base;
  float ring_tan[kMaxRings];
  float pool_tan[kMaxPool];
  double *S;                     // kValPlanes planes
  double *D;                     // kDiffPlanes planes
  unsigned long long *npix;      // per region
  double *sums;                  // per region
  double *out;                   // per region: HVSQ
  float *d_alt;                  // or null
  long long plane;               // (H + 1) * (W + 1)
};

__device__ __forceinline__ float dist2(const HvsqArgs &a, int x, int y) {
  const float dx = __fsub_rn(__fadd_rn((float)x, 0.5f), a.gx);
  const float dy = __fsub_rn(__fadd_rn((float)y, 0.5f), a.gy);
  return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

__device__ __forceinline__ int count_reached(float d2, float focal, const float *tan_, int n) {
  int c = 0;
  for (int j = 0; j < n; ++j) {
    const float R = __fmul_rn(focal, tan_[j]);
    c += d2 >= __fmul_rn(R, R) ? 1 : 0;
  }
  return c;
}

// One warp per (image row, channel): the channel's 4 values of each pixel
// (a - 1/2, its square, r - 1/2, its square), prefix-summed along the row
// into the 4 planes at (y + 1, x + 1), 256 pixels at a time: lane l sums
// pixels 8l .. 8l + 7 of the chunk in order, a warp scan of the 32 lane
// totals gives each lane its offset (FP64 adds are scarce on this GPU: about
// 2.5 per value instead of the 6 of a shuffle scan per value).  The region
// count is taken by the channel-0 warps.
constexpr int kRowRun = 8;

// One block of three warps per image row (warp c: channel c).  Each chunk
// of 256 pixels of both images is first staged in shared memory with
// coalesced loads (channel-planar, 9 floats per 8 pixels so that the lanes'
// runs fall in different banks); then lane l sums pixels 8l .. 8l + 7 in
// order and a warp scan of the lane totals gives the prefixes.
constexpr int kRowChunk = 32 * kRowRun;              // pixels per chunk
constexpr int kRowPad = kRowChunk / 8 * 9;           // padded floats per channel

__global__ void __launch_bounds__(96) k_hvsq_rows(HvsqArgs a) {
  __shared__ float s_a[3][kRowPad], s_r[3][kRowPad];
  __shared__ double s_out[3][kRowPad];   // one quantity's prefixes of the chunk, per warp
  const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
  const int y = blockIdx.x;
  const int W1 = a.W + 1;
  double *P0 = a.S + (4 * c) * a.plane + (long long)(y + 1) * W1 + 1;
  double carry[4] = {0.0, 0.0, 0.0, 0.0};
  uint32_t cnt[kMaxRings + 1] = {};   // this lane's pixels per region (channel-0 warp)
  const float *arow = a.alt + 3LL * y * a.W, *rrow = a.ref + 3LL * y * a.W;
  for (int x0 = 0; x0 < a.W; x0 += kRowChunk) {
    const int n3 = 3 * min(kRowChunk, a.W - x0);
    __syncthreads();   // the previous chunk is read
    for (int q = threadIdx.x; q < 3 * kRowChunk; q += 96) {
      const int px = q / 3, ch = q - 3 * px;
      const int sidx = px + (px >> 3);
      s_a[ch][sidx] = q < n3 ? arow[3LL * x0 + q] : 0.5f;
      s_r[ch][sidx] = q < n3 ? rrow[3LL * x0 + q] : 0.5f;
    }
    __syncthreads();
    const int xs = x0 + lane * kRowRun;
    double run[4][kRowRun];
    double tot[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int u = 0; u < kRowRun; ++u) {
      const int x = xs + u;
      const int sidx = lane * 9 + u;   // (8 lane + u) + (8 lane + u) / 8
      double v0 = 0.0, v2 = 0.0;
      if (x < a.W) {
        v0 = (double)s_a[c][sidx] - 0.5;
        v2 = (double)s_r[c][sidx] - 0.5;
        if (c == 0) {
          const int g = count_reached(dist2(a, x, y), a.focal, a.ring_tan, a.n_rings);
#pragma unroll
          for (int k = 0; k <= kMaxRings; ++k) cnt[k] += g == k ? 1u : 0u;
        }
      }
      tot[0] += v0;
      tot[1] += v0 * v0;
      tot[2] += v2;
      tot[3] += v2 * v2;
#pragma unroll
      for (int q = 0; q < 4; ++q) run[q][u] = tot[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double incl = tot[q];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const double off = carry[q] + (incl - tot[q]);
      // through shared memory, so that the global writes are coalesced
#pragma unroll
      for (int u = 0; u < kRowRun; ++u) s_out[c][lane * 9 + u] = run[q][u] + off;
      __syncwarp();
#pragma unroll
      for (int u = 0; u < kRowRun; ++u) {
        const int px = u * 32 + lane;
        if (x0 + px < a.W) P0[q * a.plane + x0 + px] = s_out[c][px + (px >> 3)];
      }
      __syncwarp();
      carry[q] += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  if (c == 0) {
#pragma unroll
    for (int k = 0; k <= kMaxRings; ++k) {
      uint32_t t = cnt[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0 && t) atomicAdd(&a.npix[k], (unsigned long long)t);
    }
  }
}

// In-place inclusive prefix along each row of `planes` planes (rows of
// W + 1 values): one warp per row, 256 values at a time, lane l summing
// values 8l .. 8l + 7 in order and a warp scan of the lane totals.
__global__ void k_scan_rows(double *P, int planes, int W1, int H1, long long plane) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long rows = (long long)planes * H1;
  if (warp >= rows) return;
  double *row = P + (warp / H1) * plane + (warp % H1) * (long long)W1;
  double carry = 0.0;
  for (int x0 = 0; x0 < W1; x0 += 32 * kRowRun) {
    const int xs = x0 + lane * kRowRun;
    double run[kRowRun];
    double tot = 0.0;
#pragma unroll
    for (int u = 0; u < kRowRun; ++u) {
      tot += xs + u < W1 ? row[xs + u] : 0.0;
      run[u] = tot;
    }
    double incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const double off = carry + (incl - tot);
#pragma unroll
    for (int u = 0; u < kRowRun; ++u)
      if (xs + u < W1) row[xs + u] = run[u] + off;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
}

// In-place inclusive prefix down each column: one block of 32 x 32 threads
// per (plane, strip of 32 columns); thread (s, c) owns rows [s L, (s + 1) L)
// of column c.  Each thread sums its segment, the segment sums are scanned in
// shared memory, and each thread re-walks its segment from its offset.
constexpr int kColSegs = 32;

__global__ void __launch_bounds__(32 * kColSegs) k_scan_cols(double *P, int planes, int W1, int H1,
                                                             long long plane) {
  __shared__ double s_part[kColSegs][33];
  const int strips = (W1 + 31) / 32;
  const int pl = blockIdx.x / strips, strip = blockIdx.x % strips;
  const int c = threadIdx.x & 31, sg = threadIdx.x >> 5;
  const int x = strip * 32 + c;
  const int L = (H1 + kColSegs - 1) / kColSegs;
  const int y0 = min(H1, sg * L), y1 = min(H1, y0 + L);
  double *col = P + (long long)pl * plane + x;
  double sum = 0.0;
  if (x < W1)
    for (int y = y0; y < y1; ++y) sum += col[(long long)y * W1];
  s_part[sg][c] = sum;
  __syncthreads();
  double acc = 0.0;
  for (int q = 0; q < sg; ++q) acc += s_part[q][c];
  if (x < W1)
    for (int y = y0; y < y1; ++y) {
      acc += col[(long long)y * W1];
      col[(long long)y * W1] = acc;
    }
  (void)planes;
}

__device__ __forceinline__ double box(const double *T, int W1, int x0, int y0, int x1, int y1) {
  // sum over [x0, x1] x [y0, y1] of the values stored at (y + 1, x + 1)
  return T[(long long)(y1 + 1) * W1 + (x1 + 1)] - T[(long long)y0 * W1 + (x1 + 1)] -
         T[(long long)(y1 + 1) * W1 + x0] + T[(long long)y0 * W1 + x0];
}

constexpr int kStatThreads = 256;

template <bool GRAD>
__global__ void __launch_bounds__(kStatThreads) k_hvsq_stats(HvsqArgs a) {
  __shared__ double s_sum[kStatThreads / 32][kMaxRings + 1];
  __shared__ double s_w[kMaxRings + 1];   // 1 / pixels of each region
  if (threadIdx.x <= kMaxRings)
    s_w[threadIdx.x] = a.npix[threadIdx.x] ? 1.0 / (double)a.npix[threadIdx.x] : 0.0;
  __syncthreads();
  double acc[kMaxRings + 1];
#pragma unroll
  for (int k = 0; k <= kMaxRings; ++k) acc[k] = 0.0;
  const long long P = (long long)a.W * a.H;
  const int W1 = a.W + 1;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / a.W), x = (int)(i - (long long)y * a.W);
    const float d2 = dist2(a, x, y);
    const int g = count_reached(d2, a.focal, a.ring_tan, a.n_rings);
    const int r = a.r_base + count_reached(d2, a.focal, a.pool_tan, a.n_pool);
    const int x0 = max(0, x - r), x1 = min(a.W - 1, x + r);
    const int y0 = max(0, y - r), y1 = min(a.H - 1, y + r);
    const double inv_n = 1.0 / ((double)(x1 - x0 + 1) * (double)(y1 - y0 + 1));
    const double w = s_w[g];
    double term = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // rounded products (no contraction into the differences below), so
      // that equal statistics give exactly zero
      const double ma = __dmul_rn(box(a.S + (4 * c + 0) * a.plane, W1, x0, y0, x1, y1), inv_n);
      const double qa = __dmul_rn(box(a.S + (4 * c + 1) * a.plane, W1, x0, y0, x1, y1), inv_n);
      const double mr = __dmul_rn(box(a.S + (4 * c + 2) * a.plane, W1, x0, y0, x1, y1), inv_n);
      const double qr = __dmul_rn(box(a.S + (4 * c + 3) * a.plane, W1, x0, y0, x1, y1), inv_n);
      // std = var / sqrt(var), and 1 / std = rsqrt(var) for the gradient
      const double va = fmax(qa - ma * ma, 0.0), vr = fmax(qr - mr * mr, 0.0);
      const double ia = va > 0.0 ? rsqrt(va) : 0.0;
      const double sa = va * ia;
      const double sr = vr > 0.0 ? vr * rsqrt(vr) : 0.0;
      const double dm = ma - mr, ds = sa - sr;
      term += dm * dm + ds * ds;
      if (GRAD) {
        // d/dx_q of w term_i for q in the box: A + (x_q - 1/2) B
        double A = 2.0 * w * dm * inv_n, B = 0.0;
        if (sa > 0.0) {
          B = 2.0 * w * ds * inv_n * ia;
          A -= B * ma;
        }
        double *DA = a.D + (2 * c) * a.plane, *DB = a.D + (2 * c + 1) * a.plane;
        const long long c00 = (long long)y0 * W1 + x0, c01 = (long long)y0 * W1 + (x1 + 1);
        const long long c10 = (long long)(y1 + 1) * W1 + x0, c11 = (long long)(y1 + 1) * W1 + (x1 + 1);
        atomicAdd(DA + c00, A);
        atomicAdd(DA + c01, -A);
        atomicAdd(DA + c10, -A);
        atomicAdd(DA + c11, A);
        if (B != 0.0) {
          atomicAdd(DB + c00, B);
          atomicAdd(DB + c01, -B);
          atomicAdd(DB + c10, -B);
          atomicAdd(DB + c11, B);
        }
      }
    }
#pragma unroll
    for (int k = 0; k <= kMaxRings; ++k) acc[k] += g == k ? term : 0.0;
  }
  // per region: warp sums, then the block's, then one global add
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k <= kMaxRings; ++k) {
    double t = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) s_sum[wid][k] = t;
  }
  __syncthreads();
  if (threadIdx.x <= a.n_rings) {
    double t = 0.0;
    for (int q = 0; q < kStatThreads / 32; ++q) t += s_sum[q][threadIdx.x];
    if (t != 0.0) atomicAdd(&a.sums[threadIdx.x], t);
  }
}

__global__ void k_hvsq_grad(HvsqArgs a) {
  const long long P = (long long)a.W * a.H;
  const int W1 = a.W + 1;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / a.W), x = (int)(i - (long long)y * a.W);
    const long long o = (long long)y * W1 + x;   // the prefix at (y, x): boxes covering it
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double A = a.D[(2 * c) * a.plane + o], B = a.D[(2 * c + 1) * a.plane + o];
      a.d_alt[3 * i + c] = (float)(A + ((double)a.alt[3 * i + c] - 0.5) * B);
    }
  }
}

__global__ void k_hvsq_final(HvsqArgs a) {
  const int g = threadIdx.x;
  if (g <= a.n_rings) a.out[g] = a.npix[g] ? a.sums[g] / (double)a.npix[g] : 0.0;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace gs

extern "C" size_t gs_hvsq_scratch_size(int32_t width, int32_t height) {
  using namespace gs;
  if (width <= 0 || height <= 0) return 0;
  const size_t plane = (size_t)(width + 1) * (size_t)(height + 1);
  return align256(sizeof(double) * plane * kValPlanes) +
         align256(sizeof(double) * plane * kDiffPlanes) +
         align256((sizeof(unsigned long long) + sizeof(double)) * (kMaxRings + 1));
}

extern "C" gs_status gs_hvsq(const float *alt, const float *ref, int32_t width, int32_t height,
                             float gaze_x, float gaze_y, float focal, const float *ring_tan,
                             int32_t n_rings, const float *pool_tan, int32_t n_pool, int32_t r_base,
                             void *scratch, size_t scratch_bytes, double *hvsq_out, float *d_alt,
                             cudaStream_t stream) {
  using namespace gs;
  if (!alt || !ref || !scratch || !hvsq_out || width <= 0 || height <= 0) return GS_ERR_INVALID_ARG;
  if (n_rings < 0 || n_rings > kMaxRings || (n_rings > 0 && !ring_tan)) return GS_ERR_INVALID_ARG;
  if (n_pool < 0 || n_pool > kMaxPool || (n_pool > 0 && !pool_tan) || r_base < 0)
    return GS_ERR_INVALID_ARG;
  if (!(focal > 0.0f) || ((uintptr_t)scratch & 255) != 0) return GS_ERR_INVALID_ARG;
  if (scratch_bytes < gs_hvsq_scratch_size(width, height)) return GS_ERR_INVALID_ARG;
  if ((long long)width * height > (1ll << 31)) return GS_ERR_INVALID_ARG;
  for (int k = 0; k < n_pool; ++k)
    if (!(pool_tan[k] > 0.0f) || (k > 0 && !(pool_tan[k] >= pool_tan[k - 1]))) return GS_ERR_INVALID_ARG;
  for (int k = 0; k < n_rings; ++k)
    if (!(ring_tan[k] > 0.0f) || (k > 0 && !(ring_tan[k] > ring_tan[k - 1]))) return GS_ERR_INVALID_ARG;
  HvsqArgs a = {};
  a.alt = alt;
  a.ref = ref;
  a.W = width;
  a.H = height;
  a.gx = gaze_x;
  a.gy = gaze_y;
  a.focal = focal;
  a.n_rings = n_rings;
  a.n_pool = n_pool;
  a.r_base = r_base;
  for (int k = 0; k < n_rings; ++k) a.ring_tan[k] = ring_tan[k];
  for (int k = 0; k < n_pool; ++k) a.pool_tan[k] = pool_tan[k];
  a.plane = (long long)(width + 1) * (height + 1);
  char *base = static_cast<char *>(scratch);
  a.S = reinterpret_cast<double *>(base);
  base += align256(sizeof(double) * (size_t)a.plane * kValPlanes);
  a.D = reinterpret_cast<double *>(base);
  base += align256(sizeof(double) * (size_t)a.plane * kDiffPlanes);
  a.npix = reinterpret_cast<unsigned long long *>(base);
  a.sums = reinterpret_cast<double *>(a.npix + (kMaxRings + 1));
  a.out = hvsq_out;
  a.d_alt = d_alt;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  const long long P = (long long)width * height;
  const int grid = (int)min((P + 255) / 256, (long long)sms * 16);
  // the tables' zero first row and column, and the accumulators
  cudaError_t e = cudaMemsetAsync(a.S, 0, sizeof(double) * (size_t)a.plane * kValPlanes, stream);
  if (e == cudaSuccess && d_alt)
    e = cudaMemsetAsync(a.D, 0, sizeof(double) * (size_t)a.plane * kDiffPlanes, stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(a.npix, 0, (sizeof(unsigned long long) + sizeof(double)) * (kMaxRings + 1),
                        stream);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  const int W1 = width + 1, H1 = height + 1;
  const int strips = (W1 + 31) / 32;
  k_hvsq_rows<<<height, 96, 0, stream>>>(a);
  k_scan_cols<<<kValPlanes * strips, 32 * kColSegs, 0, stream>>>(a.S, kValPlanes, W1, H1, a.plane);
  if (d_alt) {
    k_hvsq_stats<true><<<grid, kStatThreads, 0, stream>>>(a);
    k_scan_rows<<<(int)(((long long)kDiffPlanes * H1 * 32 + 255) / 256), 256, 0, stream>>>(a.D, kDiffPlanes, W1, H1, a.plane);
    k_scan_cols<<<kDiffPlanes * strips, 32 * kColSegs, 0, stream>>>(a.D, kDiffPlanes, W1, H1, a.plane);
    k_hvsq_grad<<<grid, 256, 0, stream>>>(a);
  } else {
    k_hvsq_stats<false><<<grid, kStatThreads, 0, stream>>>(a);
  }
  k_hvsq_final<<<1, 32, 0, stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
