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

// Whether a point of quality bound (or model level) m takes part at level
// l: nested subsets (Sec. 4.2) use the points with m >= l; with a separate
// model per level (Sec. 4.1, main pipeline) level l uses the points of
// model l only.
__device__ __forceinline__ bool takes_part(int m, int l, bool disjoint) {
  return disjoint ? m == l : m >= l;
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

// Warp layout inside a tile: each warp covers an 8 x (4 PX) block of
// pixels, PX = pixels per thread stacked 4 rows apart (16x16 tile, PX = 1:
// 2 x 4 warps; PX = 2: 2 x 2 warps).
template <int B, int PX>
struct WarpGeom {
  static constexpr int kWx = B / 8;                  // warps across
  static constexpr int kRows = 4 * PX;               // pixel rows per warp
  static constexpr int kWarps = B * B / (32 * PX);
};

// Which warps of the tile the point can reach: the bounding box of the
// region log2(alpha) >= floor - 1e-3 (an ellipse |W d|^2 <= F - floor +
// 1e-3), widened by 1e-4 relative + 1e-4 px, against each warp's pixel
// centres.  A pixel the FP32 evaluation would blend always lies inside, so
// culling never changes a decision.
template <int B, int PX>
__device__ __forceinline__ uint32_t warp_mask(float mx, float my, float4 sh, float Fmax) {
  using G = WarpGeom<B, PX>;
  const float r2 = Fmax - kLog2AlphaMin + 1e-3f;
  if (!(r2 > 0.0f)) return 0u;
  const float det = fabsf(sh.x * sh.w - sh.y * sh.z);
  const float sr = sqrtf(r2) / det;
  const float hx = sr * sqrtf(sh.y * sh.y + sh.w * sh.w) * 1.0001f + 1e-4f;
  const float hy = sr * sqrtf(sh.x * sh.x + sh.z * sh.z) * 1.0001f + 1e-4f;
  uint32_t mask = 0u;
#pragma unroll
  for (int w = 0; w < G::kWarps; ++w) {
    const float x0 = 8.0f * (w % G::kWx) + 0.5f, y0 = (float)(G::kRows * (w / G::kWx)) + 0.5f;
    const bool hit = (mx - hx <= x0 + 7.0f) && (mx + hx >= x0) &&
                     (my - hy <= y0 + (float)(G::kRows - 1)) && (my + hy >= y0);
    mask |= hit ? (1u << w) : 0u;
  }
  return mask;
}

// Exact version of warp_mask: the point can reach warp w only if the
// minimum of s(p) = |W (p - mu)|^2 over the rectangle spanned by the warp's
// pixel centres is at most F - floor (+1e-3 + 1e-4 relative slack).  The
// minimum of this convex quadratic is 0 inside, else on an edge, where it is
// a 1D quadratic minimised in closed form and clamped to the edge.
template <int B, int PX>
__device__ __forceinline__ uint32_t warp_mask_exact(float mx, float my, float4 sh, float Fmax) {
  using G = WarpGeom<B, PX>;
  const float r2 = Fmax - kLog2AlphaMin;
  if (!(r2 > -1e-3f)) return 0u;
  const float lim = r2 + 1e-3f + 1e-4f * fabsf(r2);
  const float Qa = sh.x * sh.x + sh.z * sh.z;
  const float Qb = sh.x * sh.y + sh.z * sh.w;
  const float Qc = sh.y * sh.y + sh.w * sh.w;
  const float ia = 1.0f / Qa, ic = 1.0f / Qc;
  auto f = [&](float dx, float dy) { return Qa * dx * dx + 2.0f * Qb * dx * dy + Qc * dy * dy; };
  uint32_t mask = 0u;
#pragma unroll
  for (int w = 0; w < G::kWarps; ++w) {
    const float x0 = 8.0f * (w % G::kWx) + 0.5f, x1 = x0 + 7.0f;
    const float y0 = (float)(G::kRows * (w / G::kWx)) + 0.5f, y1 = y0 + (float)(G::kRows - 1);
    float best;
    if (mx >= x0 && mx <= x1 && my >= y0 && my <= y1) {
      best = 0.0f;
    } else {
      // vertical edges x = x0, x1: dy* = -Qb dx / Qc, clamped
      float dxa = x0 - mx, dxb = x1 - mx;
      float dya = fminf(fmaxf(-Qb * dxa * ic, y0 - my), y1 - my);
      float dyb = fminf(fmaxf(-Qb * dxb * ic, y0 - my), y1 - my);
      // horizontal edges y = y0, y1
      float dyc = y0 - my, dyd = y1 - my;
      float dxc = fminf(fmaxf(-Qb * dyc * ia, x0 - mx), x1 - mx);
      float dxd = fminf(fmaxf(-Qb * dyd * ia, x0 - mx), x1 - mx);
      best = fminf(fminf(f(dxa, dya), f(dxb, dyb)), fminf(f(dxc, dyc), f(dxd, dyd)));
    }
    mask |= best * 0.9999f <= lim ? (1u << w) : 0u;
  }
  return mask;
}

// A pair of FP32 values in one 64-bit register pair, and the paired FP32
// fused multiply-add of sm_100-family GPUs on it: two correctly rounded
// fmaf results for one issued instruction.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}

__device__ __forceinline__ void f2_unpack(unsigned long long v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Evaluation record of one point in a tile: whitened offsets t = W p + c
// (p the tile-local pixel centre), so t = W (p - mu) with c = -W mu.  The
// two rows of W are interleaved so that (t1, t2) is one paired FMA chain:
//   a = (w1x, w2x, w1y, w2y), b = (c1, c2, F - floor, warp mask bits)
__device__ __forceinline__ void make_eval(float mx, float my, float4 sh, float F, uint32_t mask,
                                          float4 &a, float4 &b) {
  const float c1 = -__fmaf_rn(sh.x, mx, __fmul_rn(sh.y, my));
  const float c2 = -__fmaf_rn(sh.z, mx, __fmul_rn(sh.w, my));
  a = make_float4(sh.x, sh.z, sh.y, sh.w);
  b = make_float4(c1, c2, __fsub_rn(F, kLog2AlphaMin), __uint_as_float(mask));
}

// |t|^2 at the pixel whose centre coordinates are packed twice in px2 =
// (px, px) and py2 = (py, py):
//   t1 = fma(w1x, px, fma(w1y, py, c1)),  t2 = fma(w2x, px, fma(w2y, py, c2)),
//   s = fma(t1, t1, t2 * t2).
// The point can blend iff s <= F - floor, and then alpha = min(0.99, 2^(F - s)).
__device__ __forceinline__ float eval_s2(unsigned long long px2, unsigned long long py2,
                                         float4 a, float4 b, float &t1, float &t2) {
  const unsigned long long in = f2_fma(f2_pack(a.z, a.w), py2, f2_pack(b.x, b.y));
  f2_unpack(f2_fma(f2_pack(a.x, a.y), px2, in), t1, t2);
  return __fmaf_rn(t1, t1, __fmul_rn(t2, t2));
}

__device__ __forceinline__ float eval_s(float px, float py, float4 a, float4 b, float &t1,
                                        float &t2) {
  return eval_s2(f2_pack(px, px), f2_pack(py, py), a, b, t1, t2);
}

}  // namespace gs
