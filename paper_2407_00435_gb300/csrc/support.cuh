// support.cuh -- opacity-aware tight support of a projected point: which
// tiles of its 3-sigma rectangle can hold a pixel with alpha >= 1/255.
//
// alpha = o exp(-q/2) with q = (p - mu)^T Sigma'^-1 (p - mu), so a pixel can
// blend the point only inside the ellipse E: q <= 2 ln(255 o).  E is
// enlarged to q <= tau, tau an upper bound of 2 ln(255 o_max) (o_max: the
// largest opacity any level composites the point with):
//   255 o = m 2^e, m in [1, 2):   ln(255 o) <= e ln2_up + (m - 1)
// (ln m <= m - 1; ln2_up is the float nearest ln 2, which lies above it),
// plus a relative and an absolute slack of 2^-10 that absorb the rounding of
// the renderer's own evaluation of alpha and of the interval below.
//
// Tile (x, y) is kept if the rectangle spanned by its pixel centres,
// [xB + 0.5, xB + B - 0.5] x [yB + 0.5, yB + B - 0.5], meets E.  Per tile row
// the strip [yB + 0.5, yB + B - 0.5] cuts E in a convex set whose shadow on
// the x axis is one interval [xl, xr]: its ends are E's leftmost / rightmost
// points when they lie in the strip, else where the nearer strip edge
// crosses E.  With Sigma' = [[a, b], [b, c]], det = a c - b^2:
//   E's extent       |dx| <= sqrt(tau a),  |dy| <= sqrt(tau c)
//   rightmost point  (sqrt(tau a), b sqrt(tau a) / a)
//   on the line dy   dx = (b dy +- sqrt(det (c tau - dy^2))) / c,
// the divisions taken as products with the rounded reciprocals 1/a, 1/c.
// The kept columns of the row are the tiles whose pixel-centre span meets
// [u + xl, u + xr].  Every operation is an explicitly rounded FP32
// operation in a fixed order, so the projection (which counts the pairs)
// and the emit (which writes them) take the same decision whatever their
// compile flags, and so does the FP32 mode of the oracle.  The image does
// not change: a dropped tile holds no pixel that could blend the point.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gs {

// Upper bound of 2 ln(255 o) plus slack; negative when 255 o <= 1 (no pixel
// can reach the alpha floor).
__device__ __forceinline__ float tight_tau(float o) {
  const float x = __fmul_rn(255.0f, o);
  if (!(x > 1.0f)) return -1.0f;
  const uint32_t bits = __float_as_uint(x);
  const int e = (int)((bits >> 23) & 0xffu) - 127;                   // x = m 2^e
  const float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);  // m in [1, 2)
  float t = __fmul_rn((float)e, 0.693147182f);
  t = __fadd_rn(t, __fsub_rn(m, 1.0f));
  t = __fmul_rn(t, 2.0f);
  const float sl = __fmul_rn(t, 0.0009765625f);
  t = __fadd_rn(t, sl);
  t = __fadd_rn(t, 0.0009765625f);
  return t;
}

// Per-item quantities of the row test (each computed exactly as the
// definition does, once per item instead of once per row).
struct SuppPre {
  float u, v, b, ic, det, ct, xe, ye, dys;
  bool any;   // tau >= 0
};

__device__ __forceinline__ SuppPre supp_prep(float4 s0, float2 s1) {
  SuppPre p;
  const float a = s0.z, c = s1.x, tau = s1.y;
  p.u = s0.x;
  p.v = s0.y;
  p.b = s0.w;
  p.ic = __frcp_rn(c);
  p.any = tau >= 0.0f;
  p.det = __fsub_rn(__fmul_rn(a, c), __fmul_rn(p.b, p.b));
  p.ye = __fsqrt_rn(__fmul_rn(tau, c));
  p.xe = __fsqrt_rn(__fmul_rn(tau, a));
  p.dys = __fmul_rn(__fmul_rn(p.b, p.xe), __frcp_rn(a));   // dy of E's rightmost point
  p.ct = __fmul_rn(c, tau);
  return p;
}

// One end of the strip's cut through E: on the line dy = yb, the root
// (b yb + sgn sqrt(det (c tau - yb^2))) (1/c).
__device__ __forceinline__ float strip_end(const SuppPre &p, float yb, float sgn) {
  const float arg = fmaxf(__fmul_rn(p.det, __fsub_rn(p.ct, __fmul_rn(yb, yb))), 0.0f);
  return __fmul_rn(__fadd_rn(__fmul_rn(p.b, yb), __fmul_rn(sgn, __fsqrt_rn(arg))), p.ic);
}

// Columns [xa, xb] (not clamped to the rectangle) of tile row `by` whose
// pixel centres can meet E.  False if the row misses E.
__device__ __forceinline__ bool row_interval(const SuppPre &p, int by, int tile, int &xa,
                                             int &xb) {
  if (!p.any) return false;
  const float dy0 = __fsub_rn(__fadd_rn((float)(by * tile), 0.5f), p.v);
  const float dy1 = __fsub_rn(__fadd_rn((float)(by * tile + tile - 1), 0.5f), p.v);
  if (dy1 < -p.ye || dy0 > p.ye) return false;
  float xr, xl;
  if (p.dys >= dy0 && p.dys <= dy1) xr = p.xe;
  else xr = strip_end(p, p.dys > dy1 ? dy1 : dy0, 1.0f);
  const float ndys = -p.dys;                        // leftmost point
  if (ndys >= dy0 && ndys <= dy1) xl = -p.xe;
  else xl = strip_end(p, ndys > dy1 ? dy1 : dy0, -1.0f);
  const float L = __fadd_rn(p.u, xl), R = __fadd_rn(p.u, xr);
  const float invB = 1.0f / (float)tile;            // tile is a power of two: exact
  float fa = ceilf(__fmul_rn(__fsub_rn(__fadd_rn(L, 0.5f), (float)tile), invB));
  float fb = floorf(__fmul_rn(__fsub_rn(R, 0.5f), invB));
  fa = fminf(fmaxf(fa, -1.0f), 65536.0f);
  fb = fminf(fmaxf(fb, -1.0f), 65536.0f);
  xa = (int)fa;
  xb = (int)fb;
  return xa <= xb;
}

// Items whose rectangle has at most kTableRows rows and kTableCols columns
// get their row intervals as a table (16 bytes: for row r, byte 2r = first
// and byte 2r + 1 = last kept column, relative to the rectangle's corner;
// first > last for an empty row), written by the pair count and read by the
// emit, so that the rows are evaluated once per item.
constexpr int kTableRows = 8;
constexpr int kTableCols = 255;

__device__ __forceinline__ bool has_table(int x0, int x1, int y0, int y1) {
  return y1 - y0 < kTableRows && x1 - x0 < kTableCols;
}

// Items the emit leaves to its large-item kernel: more than kBigItem pairs,
// or (when the emit reads row tables: tight support or foveation) a
// rectangle without a table.
constexpr uint32_t kBigItem = 64;
static_assert(kBigItem < 128, "the emit's byte-packed row prefixes");

__device__ __forceinline__ bool big_item(uint32_t cnt, bool table, bool small) {
  return cnt > 0 && (cnt > kBigItem || (table && !small));
}

// Columns [la, lb] of global tile row `grow` whose tile level is <= m (the
// foveation filter keeps a pair iff tile level <= m).  A tile's level is a
// non-decreasing function of the smallest gaze distance of its pixels,
// which along a row of tiles first falls and then rises, so these columns
// form one interval.  Table entry: first | last << 16, first > last if none.
__device__ __forceinline__ void level_row(const uint32_t *rows, long long grow, int m, int &la,
                                          int &lb) {
  if (m < 1) {
    la = 1;
    lb = 0;
    return;
  }
  const uint32_t e = rows[grow * GS_MAX_LEVELS + (m > GS_MAX_LEVELS ? GS_MAX_LEVELS : m) - 1];
  la = (int)(e & 0xffffu);
  lb = (int)(e >> 16);
}

// Row r of a table: columns [x0 + first, x0 + last].
__device__ __forceinline__ void table_row(uint4 tb, int r, int &first, int &last) {
  const uint32_t w = r < 2 ? tb.x : r < 4 ? tb.y : r < 6 ? tb.z : tb.w;
  const uint32_t h = (w >> (16 * (r & 1))) & 0xffffu;
  first = (int)(h & 0xffu);
  last = (int)(h >> 8);
}

}  // namespace gs
