// raster.cuh -- the per-(pixel, point) evaluation shared by the forward and
// backward rasterizers, so that both take exactly the same alpha-floor and
// stop decisions.  Every rounding step is explicit (no implicit
// contraction), so inlining it into different kernels yields identical
// results.
#pragma once

#include <cuda_runtime.h>

#include "gs_internal.cuh"

namespace gs {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// log2(alpha) before the clamp, for a pixel at tile-local (px, py), a point
// with tile-local mean mu, whitening rows sh = (w1x, w1y, w2x, w2y) and
// F = log2(opacity):  F - t1^2 - t2^2 with t = W (p - mu).
__device__ __forceinline__ float log2_alpha(float px, float py, float2 mu, float4 sh, float F,
                                            float &dx, float &dy, float &t1, float &t2) {
  dx = __fsub_rn(px, mu.x);
  dy = __fsub_rn(py, mu.y);
  t1 = __fmaf_rn(dx, sh.x, __fmul_rn(dy, sh.y));
  t2 = __fmaf_rn(dx, sh.z, __fmul_rn(dy, sh.w));
  const float g = __fmaf_rn(-t1, t1, -__fmul_rn(t2, t2));
  return __fadd_rn(g, F);
}

__device__ __forceinline__ float alpha_of(float p) {
  return fminf(kAlphaMax, ex2_approx(p));
}

__device__ __forceinline__ int find_view(const ViewDev *views, int V, long long t) {
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (views[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Foveation level of a pixel, band membership and the blend weight of the
// pixel's own level (same FP32 expressions as the tile filter).
__device__ __forceinline__ void pixel_level(const ViewDev &vd, int L, float band, int x, int y,
                                            int &lvl, bool &in_band, float &wband) {
  lvl = 1;
  in_band = false;
  wband = 1.0f;
  if (!vd.fov) return;
  float dx = ((float)x + 0.5f) - vd.gx;
  float dy = ((float)y + 0.5f) - vd.gy;
  float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
  for (int k = 0; k < L - 1; ++k) {
    float Rk = vd.R[k];
    if (d2 >= __fmul_rn(Rk, Rk)) lvl++;
  }
  if (lvl >= 2 && band > 0.0f) {
    float Rb = __fadd_rn(vd.R[lvl - 2], band);
    if (d2 < __fmul_rn(Rb, Rb)) {
      in_band = true;
      wband = fminf(1.0f, fmaxf(0.0f, (sqrtf(d2) - vd.R[lvl - 2]) / band));
    }
  }
}

}  // namespace gs
