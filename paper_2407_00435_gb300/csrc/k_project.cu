// k_project.cu -- view table, foveation tile levels and the projection
// kernel (Sec. 2.1 "Projection"; Sec. 4.2 "Filtering").
//
// This translation unit is compiled with --fmad=false: the "keyed" part of
// the projection (visibility, camera depth, tile rectangle, the per-pixel
// foveation level) must be bit-identical to a plain IEEE evaluation of the
// same expressions in the same order, so no multiply-add may be contracted
// implicitly.  Where a fused multiply-add is wanted (error-free
// transformations of the value path) it is written as fmaf().
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_internal.cuh"
#include "support.cuh"
#include "tma.cuh"

namespace gs {

// --------------------------------------------------------------------------
// view table
// --------------------------------------------------------------------------
struct FovArgs {
  int32_t n_levels;
  float band;
  float ring_tan[GS_MAX_LEVELS - 1];
  const float *gaze;
  const uint8_t *view_fov;
};

__global__ void k_views(const gs_camera *cams, int V, int tile, FovArgs fa, int has_fov,
                        ViewDev *views, Hdr *hdr, long long tiles_total,
                        long long pixels_total, unsigned long long n_items) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long tb = 0, pb = 0, rb = 0;
  for (int v = 0; v < V; ++v) {
    const gs_camera c = cams[v];
    ViewDev d;
    d.W = c.width;
    d.H = c.height;
    d.tx = (c.width + tile - 1) / tile;
    d.ty = (c.height + tile - 1) / tile;
    d.tile_base = tb;
    d.pix_base = pb;
    // camera centre -R^T t
    d.ccx = -(c.R[0] * c.t[0] + c.R[3] * c.t[1] + c.R[6] * c.t[2]);
    d.ccy = -(c.R[1] * c.t[0] + c.R[4] * c.t[1] + c.R[7] * c.t[2]);
    d.ccz = -(c.R[2] * c.t[0] + c.R[5] * c.t[1] + c.R[8] * c.t[2]);
    d.limx = kClampFov * ((0.5f * (float)c.width) / c.fx);
    d.limy = kClampFov * ((0.5f * (float)c.height) / c.fy);
    d.fov = has_fov && fa.n_levels > 1 ? (fa.view_fov ? (int)fa.view_fov[v] : 1) : 0;
    d.gx = has_fov ? fa.gaze[2 * v] : 0.0f;
    d.gy = has_fov ? fa.gaze[2 * v + 1] : 0.0f;
    for (int k = 0; k < GS_MAX_LEVELS - 1; ++k)
      d.R[k] = (has_fov && k < fa.n_levels - 1) ? c.fy * fa.ring_tan[k] : 0.0f;
    d.row_base = (int32_t)rb;
    views[v] = d;
    rb += d.ty;
    tb += (long long)d.tx * d.ty;
    pb += (long long)c.width * c.height;
  }
  // the device cameras must describe the image sizes the plan was made for
  if (tb != tiles_total || pb != pixels_total) set_status(&hdr->status, GS_ERR_INVALID_ARG);
  hdr->n_items = n_items;
}

cudaError_t launch_views(const gs_plan *p, void *ws, cudaStream_t s) {
  FovArgs fa = {};
  if (p->has_fov) {
    fa.n_levels = p->fov.n_levels;
    fa.band = p->fov.band_px;
    for (int k = 0; k < GS_MAX_LEVELS - 1; ++k) fa.ring_tan[k] = p->fov.ring_tan[k];
    fa.gaze = p->fov.gaze_px;
    fa.view_fov = p->fov.view_fov;
  }
  k_views<<<1, 32, 0, s>>>(p->cams, p->V, p->tile, fa, p->has_fov, region<ViewDev>(p, ws, R_VIEWS),
                           region<Hdr>(p, ws, R_HDR), p->tiles_total, p->pixels_total,
                           (unsigned long long)p->max_visible);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// foveation level of a pixel (keyed FP32; same expressions as the oracle)
// --------------------------------------------------------------------------
__device__ __forceinline__ int pixel_need_level(const ViewDev &vd, int L, float band, int x,
                                                int y) {
  float dx = ((float)x + 0.5f) - vd.gx;
  float dy = ((float)y + 0.5f) - vd.gy;
  float d2 = dx * dx + dy * dy;
  int lvl = 1;
  for (int k = 0; k < L - 1; ++k) {
    float Rk = vd.R[k];
    if (d2 >= Rk * Rk) lvl++;
  }
  int need = lvl;
  if (lvl >= 2 && band > 0.0f) {
    float Rb = vd.R[lvl - 2] + band;
    if (d2 < Rb * Rb) need = lvl - 1;
  }
  return need;
}

// One warp per tile (four tiles per block); the tile's filter level is the
// smallest level any of its pixels needs (Sec. 4.2: a point takes part in a
// tile only if the tile's level t <= m).  A pixel's need is a non-decreasing
// function of its FP32 squared gaze distance (ring counts, then the band
// test of the inner ring), and that distance, fl(fl(dx^2) + fl(dy^2)), is
// non-decreasing in |dx| and |dy| separately; |fl(dx)| over the tile's
// columns is smallest at a column next to gx - 1/2 (clamped to the tile), and
// likewise for rows.  So the minimum over the tile is the need of that one
// pixel; the 4 x 4 pixels around it are evaluated, a margin for the rounding
// of the candidate itself.
constexpr int kLevelWarps = 4;

__global__ void __launch_bounds__(32 * kLevelWarps) k_tile_levels(const ViewDev *views, int V,
                                                                  int tile, int L, float band,
                                                                  uint8_t *tile_level,
                                                                  long long tiles_total) {
  const long long t = (long long)blockIdx.x * kLevelWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= tiles_total) return;   // (whole warps)
  // find the view by binary search over tile bases
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (views[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  const ViewDev &vd = views[lo];
  int local = (int)(t - vd.tile_base);
  int bx = local % vd.tx, by = local / vd.tx;
  int need = 255;
  if (vd.fov) {
    const int xa = bx * tile, xb = min(xa + tile, vd.W) - 1;
    const int ya = by * tile, yb = min(ya + tile, vd.H) - 1;
    if (lane < 16 && xa <= xb && ya <= yb) {
      // (clamped as floats first: a far gaze stays in int range)
      const int cx = (int)floorf(fminf(fmaxf(vd.gx - 0.5f, (float)xa - 2.0f), (float)xb + 2.0f));
      const int cy = (int)floorf(fminf(fmaxf(vd.gy - 0.5f, (float)ya - 2.0f), (float)yb + 2.0f));
      const int x = min(max(cx - 1 + (lane & 3), xa), xb);
      const int y = min(max(cy - 1 + (lane >> 2), ya), yb);
      need = pixel_need_level(vd, L, band, x, y);
    }
  } else {
    need = 1;
  }
  need = (int)__reduce_min_sync(0xffffffffu, (unsigned)need);
  if (lane == 0) tile_level[t] = (uint8_t)need;
}

// Per tile row and level m, the columns whose tile level is <= m (one
// interval, see level_row): one warp per tile row, lanes over its columns,
// first and last column per level by warp reductions.
__global__ void __launch_bounds__(32 * kLevelWarps) k_level_rows(const ViewDev *views, int V,
                                                                 const uint8_t *tile_level,
                                                                 long long rows_total,
                                                                 uint32_t *out) {
  const long long g = (long long)blockIdx.x * kLevelWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= rows_total) return;   // (whole warps)
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (views[mid].row_base <= g) lo = mid; else hi = mid - 1;
  }
  const ViewDev &vd = views[lo];
  const uint8_t *tl = tile_level + vd.tile_base + (g - vd.row_base) * vd.tx;
  unsigned first[GS_MAX_LEVELS], last[GS_MAX_LEVELS];
#pragma unroll
  for (int m = 0; m < GS_MAX_LEVELS; ++m) {
    first[m] = 0xffffu;
    last[m] = 0u;
  }
  for (int x = lane; x < vd.tx; x += 32) {
    const int lvl = tl[x];
#pragma unroll
    for (int m = 0; m < GS_MAX_LEVELS; ++m)
      if (lvl <= m + 1) {
        first[m] = min(first[m], (unsigned)x);
        last[m] = max(last[m], (unsigned)x);
      }
  }
#pragma unroll
  for (int m = 0; m < GS_MAX_LEVELS; ++m) {
    const unsigned f = __reduce_min_sync(0xffffffffu, first[m]);
    const unsigned l = __reduce_max_sync(0xffffffffu, last[m]);
    if (lane == 0) out[g * GS_MAX_LEVELS + m] = f | (l << 16);
  }
}

cudaError_t launch_tile_levels(const gs_plan *p, void *ws, cudaStream_t s) {
  if (!p->has_fov || p->tiles_total == 0) return cudaSuccess;
  k_tile_levels<<<(unsigned)((p->tiles_total + kLevelWarps - 1) / kLevelWarps), 32 * kLevelWarps, 0,
                  s>>>(region<ViewDev>(p, ws, R_VIEWS), p->V, p->tile, p->fov.n_levels,
                       p->fov.band_px, region<uint8_t>(p, ws, R_TILE_LEVEL), p->tiles_total);
  k_level_rows<<<(unsigned)((p->rows_total + kLevelWarps - 1) / kLevelWarps), 32 * kLevelWarps, 0,
                 s>>>(region<ViewDev>(p, ws, R_VIEWS), p->V, region<uint8_t>(p, ws, R_TILE_LEVEL),
                      p->rows_total, region<uint32_t>(p, ws, R_LEVEL_ROWS));
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// projection
// --------------------------------------------------------------------------
struct ProjArgs {
  long long n;
  int aligned16;               // every parameter array starts on 16 bytes
  int V, S, tile;
  const float *means, *scales, *quats, *opac, *sh;
  const gs_camera *cams;
  const ViewDev *views;
  const uint8_t *tile_level;   // null unless foveated
  const uint8_t *bound_m;      // null unless foveated
  Hdr *hdr;
  long long max_visible;
  float4 *rec_mean, *rec_shape, *rec_color, *rec_rest;
  uint32_t *rec_depth, *rec_count, *rec_gid, *rec_view;
  uint2 *rec_rect;
  uint8_t *rec_m;
  // opacity-aware tight support (null records = 3-sigma rectangle only)
  float4 *rec_supp;             // (u, v, a, b)
  float2 *rec_supp2;            // (c, tau)
  uint4 *rec_emit;               // emit records, 2 per slot (see k_count_pairs)
  uint32_t *rec_cbig;            // count | large-item flag << 31 (see k_count_pairs)
  const uint32_t *level_rows;    // columns kept by the foveation filter, per row and level
  const float *opacity_lv;      // (L-1, N) level opacities the support must cover, or null
  int n_opacity_lv;
  int spins;                    // polls of the staging wait before it gives up
};

struct Keyed {
  float px, py, pz;      // camera-space mean (plain FP32)
  float tx, ty;          // px/pz, py/pz
  int x0, x1, y0, y1;    // inclusive tile rect
  float M[9];            // Rq diag(s)
  float j00, j02, j11, j12;
  float u, v;            // keyed 2D mean
  float a, b, cc;        // keyed 2D covariance (with low-pass)
};

// The keyed FP32 projection.  Every statement is one IEEE operation in a
// fixed order; the FP32 mode of the oracle evaluates the same expressions.
__device__ __forceinline__ bool keyed_project(const float mu[3], const float s[3],
                                              const float q[4], const gs_camera &c,
                                              int tile, int tiles_x, int tiles_y, Keyed &k) {
  const float *R = c.R;
  float px = R[0] * mu[0];
  px = px + R[1] * mu[1];
  px = px + R[2] * mu[2];
  px = px + c.t[0];
  float py = R[3] * mu[0];
  py = py + R[4] * mu[1];
  py = py + R[5] * mu[2];
  py = py + c.t[1];
  float pz = R[6] * mu[0];
  pz = pz + R[7] * mu[1];
  pz = pz + R[8] * mu[2];
  pz = pz + c.t[2];
  if (!(pz > c.znear) || !(pz < c.zfar)) return false;

  float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
  float n2 = qw * qw;
  n2 = n2 + qx * qx;
  n2 = n2 + qy * qy;
  n2 = n2 + qz * qz;
  if (n2 > 0.0f) {
    float inv = 1.0f / sqrtf(n2);
    qw = qw * inv; qx = qx * inv; qy = qy * inv; qz = qz * inv;
  } else {
    qw = 1.0f; qx = 0.0f; qy = 0.0f; qz = 0.0f;
  }
  float r[9];
  r[0] = 1.0f - 2.0f * (qy * qy + qz * qz);
  r[1] = 2.0f * (qx * qy - qw * qz);
  r[2] = 2.0f * (qx * qz + qw * qy);
  r[3] = 2.0f * (qx * qy + qw * qz);
  r[4] = 1.0f - 2.0f * (qx * qx + qz * qz);
  r[5] = 2.0f * (qy * qz - qw * qx);
  r[6] = 2.0f * (qx * qz - qw * qy);
  r[7] = 2.0f * (qy * qz + qw * qx);
  r[8] = 1.0f - 2.0f * (qx * qx + qy * qy);
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) k.M[3 * j + kk] = r[3 * j + kk] * s[kk];

  float W = (float)c.width, H = (float)c.height;
  float limx = 1.3f * ((0.5f * W) / c.fx);
  float limy = 1.3f * ((0.5f * H) / c.fy);
  float tx = px / pz;
  float ty = py / pz;
  float txc = fminf(fmaxf(tx, -limx), limx);
  float tyc = fminf(fmaxf(ty, -limy), limy);
  float xc = txc * pz;
  float yc = tyc * pz;
  float iz = 1.0f / pz;
  float iz2 = iz * iz;
  float j00 = c.fx * iz;
  float j02 = -((c.fx * xc) * iz2);
  float j11 = c.fy * iz;
  float j12 = -((c.fy * yc) * iz2);
  float T0[3], T1[3];
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    T0[kk] = j00 * R[kk] + j02 * R[6 + kk];
    T1[kk] = j11 * R[3 + kk] + j12 * R[6 + kk];
  }
  float G0[3], G1[3];
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    float g0 = T0[0] * k.M[kk];
    g0 = g0 + T0[1] * k.M[3 + kk];
    g0 = g0 + T0[2] * k.M[6 + kk];
    G0[kk] = g0;
    float g1 = T1[0] * k.M[kk];
    g1 = g1 + T1[1] * k.M[3 + kk];
    g1 = g1 + T1[2] * k.M[6 + kk];
    G1[kk] = g1;
  }
  float a = G0[0] * G0[0];
  a = a + G0[1] * G0[1];
  a = a + G0[2] * G0[2];
  a = a + 0.3f;
  float b = G0[0] * G1[0];
  b = b + G0[1] * G1[1];
  b = b + G0[2] * G1[2];
  float cc = G1[0] * G1[0];
  cc = cc + G1[1] * G1[1];
  cc = cc + G1[2] * G1[2];
  cc = cc + 0.3f;
  float det = a * cc - b * b;
  if (!(det > 0.0f)) return false;
  float mid = 0.5f * (a + cc);
  float disc = mid * mid - det;
  disc = fmaxf(0.1f, disc);
  float lam = mid + sqrtf(disc);
  float rad = ceilf(3.0f * sqrtf(lam));
  float u = c.fx * tx + c.cx;
  float v = c.fy * ty + c.cy;
  float invB = 1.0f / (float)tile;
  float x0 = floorf((u - rad) * invB);
  float x1 = floorf((u + rad) * invB);
  float y0 = floorf((v - rad) * invB);
  float y1 = floorf((v + rad) * invB);
  x0 = fmaxf(x0, 0.0f);
  y0 = fmaxf(y0, 0.0f);
  x1 = fminf(x1, (float)(tiles_x - 1));
  y1 = fminf(y1, (float)(tiles_y - 1));
  if (!(x0 <= x1) || !(y0 <= y1)) return false;
  k.px = px; k.py = py; k.pz = pz;
  k.tx = tx; k.ty = ty;
  k.x0 = (int)x0; k.x1 = (int)x1; k.y0 = (int)y0; k.y1 = (int)y1;
  k.j00 = j00; k.j02 = j02; k.j11 = j11; k.j12 = j12;
  k.u = u; k.v = v;
  k.a = a; k.b = b; k.cc = cc;
  return true;
}

// ---- error-free transformations for the value path -----------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// Compensated R_row . mu + t: returns hi + lo to about twice FP32 precision.
__device__ __forceinline__ void dot3_comp(const float *Rr, const float mu[3], float t, float &hi,
                                          float &lo) {
  float p0, e0, p1, e1, p2, e2;
  two_prod(Rr[0], mu[0], p0, e0);
  two_prod(Rr[1], mu[1], p1, e1);
  two_prod(Rr[2], mu[2], p2, e2);
  float s, es, s2, es2, s3, es3;
  two_sum(p0, p1, s, es);
  two_sum(s, p2, s2, es2);
  two_sum(s2, t, s3, es3);
  hi = s3;
  lo = ((e0 + e1) + (e2 + es)) + (es2 + es3);
}

// (fh + fl) / (zh + zl) * f + c  as hi + lo
__device__ __forceinline__ void proj_comp(float xh, float xl, float zh, float zl, float f,
                                          float c, float &uh, float &ul) {
  float q = xh / zh;
  float r = fmaf(-q, zh, xh);          // exact residual of the division
  r = r + xl;
  r = fmaf(-q, zl, r);
  float ql = r / zh;
  float p, ep;
  two_prod(f, q, p, ep);
  float s, es;
  two_sum(p, c, s, es);
  uh = s;
  ul = es + fmaf(f, ql, ep);
}

// Real SH basis (degree <= 3) at unit direction, ordered m = -l..l.
__device__ __forceinline__ void sh_basis(float x, float y, float z, int S, float Y[16]) {
  const float k1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
  const float k2a = 1.0925484305920792f;   // 1/2 sqrt(15 / pi)
  const float k2b = 0.31539156525252005f;  // 1/4 sqrt(5 / pi)
  const float k2c = 0.54627421529603959f;  // 1/4 sqrt(15 / pi)
  const float k3a = 0.59004358992664352f;  // 1/4 sqrt(35 / (2 pi))
  const float k3b = 2.8906114426405538f;   // 1/2 sqrt(105 / pi)
  const float k3c = 0.45704579946446572f;  // 1/4 sqrt(21 / (2 pi))
  const float k3d = 0.37317633259011546f;  // 1/4 sqrt(7 / pi)
  const float k3e = 1.4453057213202769f;   // 1/4 sqrt(105 / pi)
  Y[0] = 0.28209479177387814f;
  if (S > 1) {
    Y[1] = -k1 * y;
    Y[2] = k1 * z;
    Y[3] = -k1 * x;
  }
  if (S > 4) {
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = k2a * x * y;
    Y[5] = -k2a * y * z;
    Y[6] = k2b * (2.0f * zz - xx - yy);
    Y[7] = -k2a * x * z;
    Y[8] = k2c * (xx - yy);
    if (S > 9) {
      Y[9] = -k3a * y * (3.0f * xx - yy);
      Y[10] = k3b * x * y * z;
      Y[11] = -k3c * y * (4.0f * zz - xx - yy);
      Y[12] = k3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
      Y[13] = -k3c * x * (4.0f * zz - xx - yy);
      Y[14] = k3e * z * (xx - yy);
      Y[15] = -k3a * x * (xx - 3.0f * yy);
    }
  }
}

__device__ __forceinline__ bool all_finite(const float *p, int n) {
  bool ok = true;
  for (int k = 0; k < n; ++k) ok &= isfinite(p[k]);
  return ok;
}

// Padded shared-memory rows (odd strides: no bank conflicts when every
// thread reads element k of its own row).
template <int S>
struct __align__(16) ProjSmem {
  static constexpr int kSh = (S * 3) | 1;
  float mu[kProjThreads][3];     // 16-byte aligned: TMA destinations first
  float sc[kProjThreads][3];
  float qraw[kProjThreads * 4];
  float op[kProjThreads];
  // SH rows with an odd stride; the TMA copy lands unpadded at the start of
  // the same buffer and is re-laid out in place
  float sh[kProjThreads][kSh];
  float q[kProjThreads][5];
};

// Coalesced load of `cnt` consecutive rows of `width` floats from global
// `src` (row `row0`) into a padded shared array with row stride `stride`.
__device__ __forceinline__ void stage_rows(float *dst, int stride, const float *src, long long row0,
                                           int cnt, int width) {
  const long long f0 = row0 * width;
  const int total = cnt * width;
  const float *g = src + f0;
  if ((((uintptr_t)g) & 15) == 0) {
    const int n4 = total >> 2;
    const float4 *g4 = reinterpret_cast<const float4 *>(g);
    for (int v = threadIdx.x; v < n4; v += blockDim.x) {
      const float4 x = g4[v];
      const int f = v * 4;
      dst[(f / width) * stride + f % width] = x.x;
      dst[((f + 1) / width) * stride + (f + 1) % width] = x.y;
      dst[((f + 2) / width) * stride + (f + 2) % width] = x.z;
      dst[((f + 3) / width) * stride + (f + 3) % width] = x.w;
    }
    for (int f = (n4 << 2) + threadIdx.x; f < total; f += blockDim.x)
      dst[(f / width) * stride + f % width] = g[f];
  } else {
    for (int f = threadIdx.x; f < total; f += blockDim.x)
      dst[(f / width) * stride + f % width] = g[f];
  }
}

struct Rec {
  float4 mean, shape, color, rest;
  uint32_t depth;
  uint2 rect;
  uint8_t m;
};

// Full projection of one (point, view) that passed the keyed test.
template <int S>
__device__ __forceinline__ void project_value(const ProjArgs &a, const ProjSmem<S> &sm, int tid,
                                              long long i, const float mu[3],
                                              const gs_camera &cam, const ViewDev &vd,
                                              const Keyed &k, Rec &out) {
  // --- compensated 2D mean ---
  float xh, xl, yh, yl, zh, zl;
  dot3_comp(&cam.R[0], mu, cam.t[0], xh, xl);
  dot3_comp(&cam.R[3], mu, cam.t[1], yh, yl);
  dot3_comp(&cam.R[6], mu, cam.t[2], zh, zl);
  float uh, ul, vh, vl;
  proj_comp(xh, xl, zh, zl, cam.fx, cam.cx, uh, ul);
  proj_comp(yh, yl, zh, zl, cam.fy, cam.cy, vh, vl);
  // --- 2D covariance from G = J W M, whitened (eigen form) ---
  float G0[3], G1[3], T0[3], T1[3];
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    T0[kk] = fmaf(k.j02, cam.R[6 + kk], k.j00 * cam.R[kk]);
    T1[kk] = fmaf(k.j12, cam.R[6 + kk], k.j11 * cam.R[3 + kk]);
  }
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    G0[kk] = fmaf(T0[2], k.M[6 + kk], fmaf(T0[1], k.M[3 + kk], T0[0] * k.M[kk]));
    G1[kk] = fmaf(T1[2], k.M[6 + kk], fmaf(T1[1], k.M[3 + kk], T1[0] * k.M[kk]));
  }
  const float n0 = fmaf(G0[2], G0[2], fmaf(G0[1], G0[1], G0[0] * G0[0]));
  const float n1 = fmaf(G1[2], G1[2], fmaf(G1[1], G1[1], G1[0] * G1[0]));
  const float aa = n0 + kLowpass, cc = n1 + kLowpass;
  const float bb = fmaf(G0[2], G1[2], fmaf(G0[1], G1[1], G0[0] * G1[0]));
  // det(G G^T + 0.3 I) = sum of squared 2x2 minors + 0.3 (|G0|^2 + |G1|^2) + 0.09
  float det = kLowpass * kLowpass + kLowpass * (n0 + n1);
#pragma unroll
  for (int p0 = 0; p0 < 3; ++p0) {
    const int p1 = (p0 + 1) % 3;
    const float w = G0[p1] * G1[p0];
    const float e = fmaf(-G0[p1], G1[p0], w);
    const float f = fmaf(G0[p0], G1[p1], -w);
    const float m = f + e;
    det = fmaf(m, m, det);
  }
  const float hd = 0.5f * (aa - cc);
  const float hyp = sqrtf(fmaf(hd, hd, bb * bb));
  const float l1 = 0.5f * (aa + cc) + hyp;
  const float l2 = det / l1;
  float e1x, e1y;
  if (aa >= cc) { e1x = hd + hyp; e1y = bb; } else { e1x = bb; e1y = hyp - hd; }
  const float en = sqrtf(fmaf(e1x, e1x, e1y * e1y));
  if (en > 0.0f) { e1x = e1x / en; e1y = e1y / en; } else { e1x = 1.0f; e1y = 0.0f; }
  const float s1 = kWhiten / sqrtf(l1), s2 = kWhiten / sqrtf(l2);
  out.shape = make_float4(e1x * s1, e1y * s1, -e1y * s2, e1x * s2);
  // --- colour g(SH) at the view direction ---
  const float dx = mu[0] - vd.ccx, dy = mu[1] - vd.ccy, dz = mu[2] - vd.ccz;
  const float dn = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  const float inv = dn > 0.0f ? 1.0f / dn : 0.0f;
  float Y[16];
  sh_basis(dx * inv, dy * inv, dz * inv, S, Y);
  const float *shc = sm.sh[tid];
  float rest[3], col[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float acc = 0.0f;
#pragma unroll
    for (int kk = 1; kk < S; ++kk) acc = fmaf(shc[3 * kk + ch], Y[kk], acc);
    rest[ch] = acc;
    col[ch] = fmaxf(0.0f, fmaf(shc[ch], Y[0], acc) + kShOffset);
  }
  out.mean = make_float4(uh, vh, ul, vl);
  out.color = make_float4(col[0], col[1], col[2], log2f(sm.op[tid]));
  out.rest = make_float4(rest[0], rest[1], rest[2], 0.0f);
  out.depth = __float_as_uint(k.pz);
  out.rect = make_uint2((uint32_t)k.x0 | ((uint32_t)k.x1 << 16), (uint32_t)k.y0 | ((uint32_t)k.y1 << 16));
  out.m = a.tile_level ? a.bound_m[i] : 0;
}

// Tile pairs of every visible item: the rectangle's tiles that pass the
// foveation filter (tile level <= m: one interval per row, from the level
// rows) and, with the tight support, lie in their row's interval.  Items
// whose rectangle has at most kTableRows rows get their row intervals as a
// table for the emit; their rows are evaluated warp-cooperatively: the rows
// of a warp's 32 items are spread over the lanes (owner found by binary
// search over the row prefix sums, its constants fetched by shuffles) and
// the per-row results meet in shared memory.  With the tight support, items
// with more rows are taken by the whole warp, one at a time, lanes over rows.
// Besides the count, every visible item gets its emit record (32 bytes, one
// sector, so the emit gathers one sector per item):
//   [0] = (global tile id of the rectangle's corner, width | rows << 16,
//          tiles per row of the item's view, count)
//   [1] = the row table (only written, and only read, for items that have one)
// and, in a compact array, the count with the large-item flag in bit 31 (what
// the offset upsweep gathers in depth order).  It also clears the counter of
// the large-item queue that the upsweep, which runs after it, fills.
constexpr int kCountThreads = 256;

__global__ void __launch_bounds__(kCountThreads) k_count_pairs(ProjArgs a) {
  __shared__ __align__(16) uint16_t s_row[kCountThreads / 32][32][kTableRows];   // xa | xb << 8
                                                                                 //   (relative)
  const long long slots = a.n * a.V;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const long long warps = (long long)gridDim.x * (kCountThreads / 32);
  const long long wid = (long long)blockIdx.x * (kCountThreads / 32) + wl;
  const bool tight = a.rec_supp != nullptr, fov = a.tile_level != nullptr;
  if (blockIdx.x == 0 && threadIdx.x == 0) a.hdr->big_count = 0u;
  // the view of slot j = i V + v, by 32-bit division where the slots allow
  // (a 64-bit remainder is a long instruction sequence)
  const bool slots32 = slots <= 0xffffffffLL;
  auto view_of = [&](long long jj) -> int {
    if (a.V == 1) return 0;
    return slots32 ? (int)((uint32_t)jj % (uint32_t)a.V) : (int)(jj % a.V);
  };
  for (long long base = wid * 32; base < slots; base += warps * 32) {
    const long long j = base + lane;
    const int vj = view_of(j);
    // every record the item may need, loaded at once (invisible slots hold
    // stale values that are never used): one round trip instead of a chain
    const bool in = j < slots;
    const uint32_t dkey = in ? a.rec_depth[j] : 0xffffffffu;
    const uint2 rr = in ? a.rec_rect[j] : make_uint2(0u, 0u);
    float4 sp = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 sp2 = make_float2(0.f, 0.f);
    if (tight && in) {
      sp = a.rec_supp[j];
      sp2 = a.rec_supp2[j];
    }
    const int mrec = (fov && in) ? (int)a.rec_m[j] : 0;
    bool vis = false;
    int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
    if (dkey != 0xffffffffu) {
      vis = true;
      x0 = rr.x & 0xffff; x1 = rr.x >> 16; y0 = rr.y & 0xffff; y1 = rr.y >> 16;
    }
    // rows this lane's item contributes to the cooperative pass
    int rows = 0;
    uint32_t my_count = 0;
    if (vis) {
      if (!tight && !fov) {
        my_count = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
      } else if (!has_table(x0, x1, y0, y1)) {
        if (tight) {
          // many rows: counted by the whole warp below
        } else {
          // foveation filter only: one interval lookup per row
          const ViewDev &vd = a.views[vj];
          const int m = mrec;
          uint32_t pairs = 0;
          for (int y = y0; y <= y1; ++y) {
            int la, lb;
            level_row(a.level_rows, vd.row_base + y, m, la, lb);
            const int xa = max(x0, la), xb = min(x1, lb);
            if (xa <= xb) pairs += (uint32_t)(xb - xa + 1);
          }
          my_count = pairs;
        }
      } else {
        rows = y1 - y0 + 1;
      }
    }
    // per-item constants of the row test
    SuppPre pre = {};
    int m = 0, rbase = 0;
    if (rows) {
      if (tight) pre = supp_prep(sp, sp2);
      if (fov) {
        m = mrec;
        rbase = a.views[vj].row_base;
      }
    }
    // inclusive prefix of the rows over the warp
    int incl = rows;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - rows;
    for (int q0 = 0; q0 < total; q0 += 32) {
      const int q = q0 + lane;
      // owner: the first lane whose inclusive prefix exceeds q
      int L = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int e = __shfl_sync(0xffffffffu, incl, L + step - 1);
        if (e <= q) L += step;
      }
      const int oexcl = __shfl_sync(0xffffffffu, excl, L);
      const int ox0 = __shfl_sync(0xffffffffu, x0, L), ox1 = __shfl_sync(0xffffffffu, x1, L);
      const int oy0 = __shfl_sync(0xffffffffu, y0, L);
      SuppPre p = {};
      if (tight) {
        p.u = __shfl_sync(0xffffffffu, pre.u, L);
        p.v = __shfl_sync(0xffffffffu, pre.v, L);
        p.b = __shfl_sync(0xffffffffu, pre.b, L);
        p.ic = __shfl_sync(0xffffffffu, pre.ic, L);
        p.det = __shfl_sync(0xffffffffu, pre.det, L);
        p.ct = __shfl_sync(0xffffffffu, pre.ct, L);
        p.xe = __shfl_sync(0xffffffffu, pre.xe, L);
        p.ye = __shfl_sync(0xffffffffu, pre.ye, L);
        p.dys = __shfl_sync(0xffffffffu, pre.dys, L);
        p.any = __shfl_sync(0xffffffffu, (int)pre.any, L) != 0;
      }
      const int om = __shfl_sync(0xffffffffu, m, L), orb = __shfl_sync(0xffffffffu, rbase, L);
      if (q < total) {
        const int r = q - oexcl, y = oy0 + r;
        int xa = ox0, xb = ox1;
        bool any = true;
        if (tight) {
          int ia, ib;
          any = row_interval(p, y, a.tile, ia, ib);
          xa = max(xa, ia);
          xb = min(xb, ib);
        }
        if (fov) {
          int la, lb;
          level_row(a.level_rows, orb + y, om, la, lb);
          xa = max(xa, la);
          xb = min(xb, lb);
        }
        s_row[wl][L][r] = (any && xa <= xb) ? (uint16_t)((xa - ox0) | ((xb - ox0) << 8))
                                            : (uint16_t)0x00ffu;   // empty: first 255 > last 0
      }
    }
    __syncwarp();
    // tight support, rectangles without a table: the whole warp takes each
    // such item in turn, lanes over its rows
    uint32_t pending = __ballot_sync(0xffffffffu, vis && tight && !has_table(x0, x1, y0, y1));
    while (pending) {
      const int src = __ffs(pending) - 1;
      pending &= pending - 1;
      const int bx0 = __shfl_sync(0xffffffffu, x0, src), bx1 = __shfl_sync(0xffffffffu, x1, src);
      const int by0 = __shfl_sync(0xffffffffu, y0, src), by1 = __shfl_sync(0xffffffffu, y1, src);
      const float2 s1 = make_float2(__shfl_sync(0xffffffffu, sp2.x, src),
                                    __shfl_sync(0xffffffffu, sp2.y, src));
      const float4 bsp = make_float4(
          __shfl_sync(0xffffffffu, sp.x, src), __shfl_sync(0xffffffffu, sp.y, src),
          __shfl_sync(0xffffffffu, sp.z, src), __shfl_sync(0xffffffffu, sp.w, src));
      const SuppPre pb = supp_prep(bsp, s1);
      const int bm = __shfl_sync(0xffffffffu, mrec, src);
      const int brb = fov ? a.views[__shfl_sync(0xffffffffu, vj, src)].row_base : 0;
      uint32_t bpairs = 0;
      for (int y = by0 + lane; y <= by1; y += 32) {
        int xa, xb;
        if (!row_interval(pb, y, a.tile, xa, xb)) continue;
        xa = max(xa, bx0);
        xb = min(xb, bx1);
        if (fov) {
          int la, lb;
          level_row(a.level_rows, brb + y, bm, la, lb);
          xa = max(xa, la);
          xb = min(xb, lb);
        }
        if (xa <= xb) bpairs += (uint32_t)(xb - xa + 1);
      }
      for (int o = 16; o > 0; o >>= 1) bpairs += __shfl_xor_sync(0xffffffffu, bpairs, o);
      if (lane == src) my_count = bpairs;
    }
    if (rows) {
      // the item's 8 table entries in one load; rows past its last are empty
      // (first 255 > last 0)
      static_assert(kTableRows == 8, "one 16-byte load per table");
      const uint4 raw = *reinterpret_cast<const uint4 *>(&s_row[wl][lane][0]);
      uint32_t tb[4] = {raw.x, raw.y, raw.z, raw.w};
      uint32_t pairs = 0;
#pragma unroll
      for (int r = 0; r < kTableRows; ++r) {
        const int sh = 16 * (r & 1);
        uint32_t e = (tb[r >> 1] >> sh) & 0xffffu;
        if (r >= rows) e = 0x00ffu;
        const int first = (int)(e & 0xffu), last = (int)(e >> 8);
        if (first <= last) pairs += (uint32_t)(last - first + 1);
        tb[r >> 1] = (tb[r >> 1] & ~(0xffffu << sh)) | (e << sh);
      }
      my_count = pairs;
      a.rec_emit[2 * j + 1] = make_uint4(tb[0], tb[1], tb[2], tb[3]);
    }
    if (vis) {
      const ViewDev &vd = a.views[vj];
      const uint32_t corner = (uint32_t)(vd.tile_base + (long long)y0 * vd.tx + x0);
      a.rec_count[j] = my_count;
      a.rec_emit[2 * j] = make_uint4(corner, (uint32_t)(x1 - x0 + 1) | ((uint32_t)(y1 - y0 + 1) << 16),
                                     (uint32_t)vd.tx, my_count);
      const bool big = big_item(my_count, tight || fov, has_table(x0, x1, y0, y1));
      a.rec_cbig[j] = my_count | (big ? 0x80000000u : 0u);
    }
    __syncwarp();
  }
}

__device__ __forceinline__ void write_rec(const ProjArgs &a, unsigned long long j, const Rec &r,
                                          uint32_t gid, uint32_t v) {
  a.rec_mean[j] = r.mean;
  a.rec_shape[j] = r.shape;
  a.rec_color[j] = r.color;
  if (a.rec_rest) {
    a.rec_rest[j] = r.rest;
    a.rec_m[j] = r.m;
  }
  a.rec_depth[j] = r.depth;
  a.rec_rect[j] = r.rect;
  a.rec_gid[j] = gid;
  a.rec_view[j] = v;
}

// One thread per point, looping over the views.  Records live at fixed
// slots j = i * V + v (point-major): no compaction pass, so no look-back
// chain.  Invisible slots get depth key 0xffffffff (they sort after every
// visible item) and zero pairs; the number of visible items is counted with
// one atomic per block.
template <int S>
__global__ void __launch_bounds__(kProjThreads, 10) k_project(ProjArgs a) {
  __shared__ ProjSmem<S> sm;
  __shared__ uint32_t s_vis, s_nonfinite, s_dmax, s_dnmin;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_vis = 0;
    s_dmax = 0;
    s_dnmin = 0;
    s_nonfinite = 0;
  }
  __shared__ __align__(8) uint64_t s_bar;
  const long long row0 = (long long)blockIdx.x * kProjThreads;
  const int cnt_rows = (int)min((long long)kProjThreads, a.n - row0);
  // Full blocks whose source chunks are 16-byte aligned are fetched by the
  // TMA engine (cp.async.bulk, one thread issues five copies); the SH rows
  // are then re-laid out into odd-stride rows.  Other blocks load with
  // ordinary coalesced loads.
  const bool tma = cnt_rows == kProjThreads && a.aligned16;
  if (tma) {
    if (tid == 0) {
      mbar_init(&s_bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
      constexpr uint32_t bsh = kProjThreads * S * 3 * 4, b3 = kProjThreads * 3 * 4;
      constexpr uint32_t bq = kProjThreads * 4 * 4, bo = kProjThreads * 4;
      mbar_expect_tx(&s_bar, bsh + 2 * b3 + bq + bo);
      bulk_g2s(&sm.sh[0][0], a.sh + row0 * S * 3, bsh, &s_bar);
      bulk_g2s(&sm.mu[0][0], a.means + row0 * 3, b3, &s_bar);
      bulk_g2s(&sm.sc[0][0], a.scales + row0 * 3, b3, &s_bar);
      bulk_g2s(&sm.qraw[0], a.quats + row0 * 4, bq, &s_bar);
      bulk_g2s(&sm.op[0], a.opac + row0, bo, &s_bar);
    }
    const bool landed = mbar_wait_bounded(&s_bar, 0, a.spins);
    if (__syncthreads_or(!landed)) {
      // give up together: record it, wait (bounded, the full limit) for the
      // copies still in flight into this block's shared memory, then leave
      if (tid == 0) set_status(&a.hdr->status, GS_ERR_TIMEOUT);
      mbar_wait_bounded(&s_bar, 0);
      return;
    }
    // in-place re-layout of the SH rows: each thread pulls its own unpadded
    // row into registers, then writes it back with the odd stride
    float row[S * 3];
    const float *raw = &sm.sh[0][0] + tid * (S * 3);
    if constexpr ((S * 3) % 4 == 0) {
#pragma unroll
      for (int k = 0; k < S * 3; k += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(raw + k);
        row[k] = v.x; row[k + 1] = v.y; row[k + 2] = v.z; row[k + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < S * 3; ++k) row[k] = raw[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < S * 3; ++k) sm.sh[tid][k] = row[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) sm.q[tid][k] = sm.qraw[tid * 4 + k];
  } else {
    stage_rows(&sm.sh[0][0], ProjSmem<S>::kSh, a.sh, row0, cnt_rows, S * 3);
    stage_rows(&sm.mu[0][0], 3, a.means, row0, cnt_rows, 3);
    stage_rows(&sm.sc[0][0], 3, a.scales, row0, cnt_rows, 3);
    stage_rows(&sm.q[0][0], 5, a.quats, row0, cnt_rows, 4);
    stage_rows(&sm.op[0], 1, a.opac, row0, cnt_rows, 1);
  }
  __syncthreads();
  // per point: finite parameters, tight-support tau (the largest opacity
  // any level composites the point with; one value shared by its views)
  __shared__ uint8_t s_fin[kProjThreads];
  __shared__ float s_tau[kProjThreads];
  if (tid < cnt_rows) {
    float mu[3], sc[3], q[4];
#pragma unroll
    for (int k = 0; k < 3; ++k) { mu[k] = sm.mu[tid][k]; sc[k] = sm.sc[tid][k]; }
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = sm.q[tid][k];
    const bool fin = all_finite(mu, 3) && all_finite(sc, 3) && all_finite(q, 4) &&
                     isfinite(sm.op[tid]) && all_finite(sm.sh[tid], S * 3);
    if (!fin) atomicAdd(&s_nonfinite, (uint32_t)a.V);
    float tau = 0.0f;
    if (a.rec_supp) {
      float o_max = sm.op[tid];
      for (int l = 0; l < a.n_opacity_lv; ++l)
        o_max = fmaxf(o_max, a.opacity_lv[(long long)l * a.n + row0 + tid]);
      tau = tight_tau(o_max);
    }
    s_fin[tid] = fin ? 1 : 0;
    s_tau[tid] = tau;
  }
  __syncthreads();
  // items (point, view) of the block, consecutive threads on consecutive
  // slots j = i V + v (coalesced record writes; one view: one point each)
  uint32_t nvis = 0, dmax = 0, dnmin = 0;   // visible items; largest depth key and complement
  const int items = cnt_rows * a.V;
  for (int k = tid; k < items; k += kProjThreads) {
    const int pl = a.V == 1 ? k : k / a.V;
    const int v = k - pl * a.V;
    const long long i = row0 + pl;
    float mu[3], sc[3], q[4];
#pragma unroll
    for (int c = 0; c < 3; ++c) { mu[c] = sm.mu[pl][c]; sc[c] = sm.sc[pl][c]; }
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = sm.q[pl][c];
    const bool fin = s_fin[pl] != 0;
    {
      const long long j = i * a.V + v;
      const gs_camera cam = a.cams[v];
      const ViewDev &vd = a.views[v];
      Keyed kk;
      if (fin && keyed_project(mu, sc, q, cam, a.tile, vd.tx, vd.ty, kk)) {
        if (a.rec_supp) {
          // keyed mean and covariance, tau
          a.rec_supp[j] = make_float4(kk.u, kk.v, kk.a, kk.b);
          a.rec_supp2[j] = make_float2(kk.cc, s_tau[pl]);
        }
        Rec r;
        project_value<S>(a, sm, pl, i, mu, cam, vd, kk, r);
        write_rec(a, (unsigned long long)j, r, (uint32_t)i, (uint32_t)v);
        ++nvis;
        dmax = max(dmax, r.depth);
        dnmin = max(dnmin, ~r.depth);
      } else {
        a.rec_depth[j] = 0xffffffffu;
        a.rec_count[j] = 0u;
      }
    }
  }
  if (nvis) {
    atomicAdd(&s_vis, nvis);
    atomicMax(&s_dmax, dmax);
    atomicMax(&s_dnmin, dnmin);
  }
  __syncthreads();
  if (tid == 0) {
    if (s_vis) {
      atomicAdd(&a.hdr->n_visible, (unsigned long long)s_vis);
      atomicMax(&a.hdr->depth_max, s_dmax);
      atomicMax(&a.hdr->depth_nmin, s_dnmin);
    }
    if (s_nonfinite) atomicAdd(&a.hdr->n_nonfinite, (unsigned long long)s_nonfinite);
  }
}

static ProjArgs make_proj_args(const gs_plan *p, void *ws) {
  ProjArgs a;
  a.n = p->n;
  a.V = p->V;
  a.S = (p->sh_degree + 1) * (p->sh_degree + 1);
  a.tile = p->tile;
  a.means = p->scene.means;
  a.scales = p->scene.scales;
  a.quats = p->scene.quats;
  a.opac = p->scene.opacities;
  a.sh = p->scene.sh;
  a.cams = p->cams;
  auto al16 = [](const void *q) { return ((uintptr_t)q & 15) == 0; };
  a.aligned16 = al16(a.means) && al16(a.scales) && al16(a.quats) && al16(a.opac) && al16(a.sh);
  a.views = region<ViewDev>(p, ws, R_VIEWS);
  a.tile_level = p->has_fov ? region<uint8_t>(p, ws, R_TILE_LEVEL) : nullptr;
  a.bound_m = p->has_fov ? p->fov.bound_m : nullptr;
  a.hdr = region<Hdr>(p, ws, R_HDR);
  a.max_visible = p->max_visible;
  a.rec_mean = region<float4>(p, ws, R_REC_MEAN);
  a.rec_shape = region<float4>(p, ws, R_REC_SHAPE);
  a.rec_color = region<float4>(p, ws, R_REC_COLOR);
  a.rec_rest = p->bytes[R_REC_REST] ? region<float4>(p, ws, R_REC_REST) : nullptr;
  a.rec_depth = region<uint32_t>(p, ws, R_REC_DEPTH);
  a.rec_count = region<uint32_t>(p, ws, R_REC_COUNT);
  a.rec_gid = region<uint32_t>(p, ws, R_REC_GID);
  a.rec_view = region<uint32_t>(p, ws, R_REC_VIEW);
  a.rec_rect = region<uint2>(p, ws, R_REC_RECT);
  a.rec_m = p->bytes[R_REC_M] ? region<uint8_t>(p, ws, R_REC_M) : nullptr;
  const bool tight = (p->flags & GS_FLAG_TIGHT) != 0;
  a.rec_supp = tight ? region<float4>(p, ws, R_REC_SUPP) : nullptr;
  a.rec_supp2 = tight ? region<float2>(p, ws, R_REC_SUPP2) : nullptr;
  a.rec_emit = region<uint4>(p, ws, R_REC_EMIT);
  a.rec_cbig = region<uint32_t>(p, ws, R_REC_CBIG);
  a.level_rows = p->has_fov ? region<uint32_t>(p, ws, R_LEVEL_ROWS) : nullptr;
  a.opacity_lv = p->has_fov ? p->fov.opacity_lv : nullptr;
  a.n_opacity_lv = a.opacity_lv ? p->fov.n_levels - 1 : 0;
  a.spins = p->wait_spins == 0 ? kSpinLimit : (p->wait_spins < 0 ? 0 : p->wait_spins);
  return a;
}

cudaError_t launch_project(const gs_plan *p, void *ws, cudaStream_t s) {
  if (p->n == 0) return cudaSuccess;
  const ProjArgs a = make_proj_args(p, ws);
  unsigned grid = (unsigned)((p->n + kProjThreads - 1) / kProjThreads);
  switch (a.S) {
    case 1: k_project<1><<<grid, kProjThreads, 0, s>>>(a); break;
    case 4: k_project<4><<<grid, kProjThreads, 0, s>>>(a); break;
    case 9: k_project<9><<<grid, kProjThreads, 0, s>>>(a); break;
    default: k_project<16><<<grid, kProjThreads, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_count_pairs(const gs_plan *p, void *ws, cudaStream_t s) {
  if (p->n == 0) return cudaSuccess;
  const ProjArgs a = make_proj_args(p, ws);
  const long long slots = p->n * p->V;
  const long long cb = (slots + kCountThreads - 1) / kCountThreads;
  k_count_pairs<<<(unsigned)(cb < 65535 ? cb : 65535), kCountThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace gs
