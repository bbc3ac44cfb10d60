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
//   fill     per pixel and channel, v = x - 1/2 and v^2 of both images into
//            12 planes of (H+1) x (W+1) (first row and column zero)
//   scan     in-place inclusive 2D prefix: summed-area tables, so that a
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

__global__ void k_hvsq_fill(HvsqArgs a) {
  const long long P = (long long)a.W * a.H;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / a.W), x = (int)(i - (long long)y * a.W);
    const int g = count_reached(dist2(a, x, y), a.focal, a.ring_tan, a.n_rings);
    atomicAdd(&a.npix[g], 1ull);
    const long long o = (long long)(y + 1) * (a.W + 1) + (x + 1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double va = (double)a.alt[3 * i + c] - 0.5, vr = (double)a.ref[3 * i + c] - 0.5;
      a.S[(4 * c + 0) * a.plane + o] = va;
      a.S[(4 * c + 1) * a.plane + o] = va * va;
      a.S[(4 * c + 2) * a.plane + o] = vr;
      a.S[(4 * c + 3) * a.plane + o] = vr * vr;
    }
  }
}

// In-place inclusive prefix along each row of `planes` planes (rows of
// W + 1 values): one warp per row, 32 values at a time with a carry.
__global__ void k_scan_rows(double *P, int planes, int W1, int H1, long long plane) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long rows = (long long)planes * H1;
  if (warp >= rows) return;
  double *row = P + (warp / H1) * plane + (warp % H1) * (long long)W1;
  double carry = 0.0;
  for (int x0 = 0; x0 < W1; x0 += 32) {
    const int x = x0 + lane;
    double v = x < W1 ? row[x] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    v += carry;
    if (x < W1) row[x] = v;
    carry = __shfl_sync(0xffffffffu, v, 31);
  }
}

// In-place inclusive prefix down each column: one thread per (plane,
// column), rows read 8 at a time.
__global__ void k_scan_cols(double *P, int planes, int W1, int H1, long long plane) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)planes * W1) return;
  double *col = P + (t / W1) * plane + (t % W1);
  double acc = 0.0;
  int y = 0;
  for (; y + 8 <= H1; y += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = col[(long long)(y + u) * W1];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      acc += v[u];
      col[(long long)(y + u) * W1] = acc;
    }
  }
  for (; y < H1; ++y) {
    acc += col[(long long)y * W1];
    col[(long long)y * W1] = acc;
  }
}

__device__ __forceinline__ double box(const double *T, int W1, int x0, int y0, int x1, int y1) {
  // sum over [x0, x1] x [y0, y1] of the values stored at (y + 1, x + 1)
  return T[(long long)(y1 + 1) * W1 + (x1 + 1)] - T[(long long)y0 * W1 + (x1 + 1)] -
         T[(long long)(y1 + 1) * W1 + x0] + T[(long long)y0 * W1 + x0];
}

constexpr int kStatThreads = 256;

template <bool GRAD>
__global__ void __launch_bounds__(kStatThreads) k_hvsq_stats(HvsqArgs a) {
  __shared__ double s_sum[kMaxRings + 1];
  if (threadIdx.x <= kMaxRings) s_sum[threadIdx.x] = 0.0;
  __syncthreads();
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
    const double n = (double)(x1 - x0 + 1) * (double)(y1 - y0 + 1);
    const double w = 1.0 / (double)a.npix[g];
    double term = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double ma = box(a.S + (4 * c + 0) * a.plane, W1, x0, y0, x1, y1) / n;
      const double qa = box(a.S + (4 * c + 1) * a.plane, W1, x0, y0, x1, y1) / n;
      const double mr = box(a.S + (4 * c + 2) * a.plane, W1, x0, y0, x1, y1) / n;
      const double qr = box(a.S + (4 * c + 3) * a.plane, W1, x0, y0, x1, y1) / n;
      const double sa = sqrt(fmax(qa - ma * ma, 0.0));
      const double sr = sqrt(fmax(qr - mr * mr, 0.0));
      const double dm = ma - mr, ds = sa - sr;
      term += dm * dm + ds * ds;
      if (GRAD) {
        // d/dx_q of w term_i for q in the box: A + (x_q - 1/2) B
        double A = 2.0 * w * dm / n, B = 0.0;
        if (sa > 0.0) {
          B = 2.0 * w * ds / (n * sa);
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
    atomicAdd(&s_sum[g], term);
  }
  __syncthreads();
  if (threadIdx.x <= a.n_rings && s_sum[threadIdx.x] != 0.0) atomicAdd(&a.sums[threadIdx.x], s_sum[threadIdx.x]);
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
  k_hvsq_fill<<<grid, 256, 0, stream>>>(a);
  k_scan_rows<<<(int)(((long long)kValPlanes * H1 * 32 + 255) / 256), 256, 0, stream>>>(a.S, kValPlanes, W1, H1, a.plane);
  k_scan_cols<<<(int)(((long long)kValPlanes * W1 + 255) / 256), 256, 0, stream>>>(a.S, kValPlanes, W1, H1, a.plane);
  if (d_alt) {
    k_hvsq_stats<true><<<grid, kStatThreads, 0, stream>>>(a);
    k_scan_rows<<<(int)(((long long)kDiffPlanes * H1 * 32 + 255) / 256), 256, 0, stream>>>(a.D, kDiffPlanes, W1, H1, a.plane);
    k_scan_cols<<<(int)(((long long)kDiffPlanes * W1 + 255) / 256), 256, 0, stream>>>(a.D, kDiffPlanes, W1, H1, a.plane);
    k_hvsq_grad<<<grid, 256, 0, stream>>>(a);
  } else {
    k_hvsq_stats<false><<<grid, kStatThreads, 0, stream>>>(a);
  }
  k_hvsq_final<<<1, 32, 0, stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
