/*
 * gs_oracle.c -- plain, slow CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  It shares no code with the CUDA path.  See
 * gs_oracle.h for the definition it implements and the paper passages it
 * follows.  Build with -O2 -ffp-contract=off (no fast-math): the keyed FP32
 * path relies on every float operation being rounded on its own.
 *
 * Parity pins live in tests/test_oracle_*.py (closed forms, brute force,
 * invariants, SciPy's spherical harmonics, finite differences).
 */
#include "gs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>


/* Readings of the constants the paper leaves to the 3DGS paper (Sec. 2.1,
 * after Eq. 1: "refer readers to Kerbl et al. for the details of f and g"). */
#define LOWPASS 0.3            /* px^2 added to the 2D covariance diagonal */
#define ALPHA_MIN (1.0 / 255.0) /* alpha floor: weaker splats are skipped */
#define ALPHA_MAX 0.99         /* alpha clamp */
#define T_MIN 1e-4             /* stop before a splat that takes T below it */
#define CLAMP_FOV 1.3          /* J uses x/z clamped to 1.3 tan(half fov) */
#define SH_OFFSET 0.5          /* colour = max(0, SH . Y + 0.5) */
#define Y00 0.28209479177387814 /* 1 / (2 sqrt(pi)) */

/* ------------------------------------------------------------------------ */
/* views and tiles                                                          */
/* ------------------------------------------------------------------------ */
static void view_tiles(const orc_cam *c, int tile, int *tx, int *ty) {
  *tx = (c->width + tile - 1) / tile;
  *ty = (c->height + tile - 1) / tile;
}

int64_t orc_total_tiles(int V, const orc_cam *cams, int tile) {
  int64_t s = 0;
  for (int v = 0; v < V; ++v) {
    int tx, ty;
    view_tiles(&cams[v], tile, &tx, &ty);
    s += (int64_t)tx * ty;
  }
  return s;
}

static int64_t tile_base(int V, const orc_cam *cams, int tile, int v) {
  (void)V;
  return orc_total_tiles(v, cams, tile);
}

static int64_t pix_base(const orc_cam *cams, int v) {
  int64_t s = 0;
  for (int u = 0; u < v; ++u) s += (int64_t)cams[u].width * cams[u].height;
  return s;
}

/* ------------------------------------------------------------------------ */
/* keyed FP32 projection: visibility, depth bits, tile rectangle            */
/*                                                                          */
/* Fixed operation order (every line one IEEE-rounded float operation, no   */
/* contraction); the CUDA projection follows the same order.                */
/* ------------------------------------------------------------------------ */
static uint32_t f32_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

/* ------------------------------------------------------------------------ */
/* opacity-aware tight support (optional)                                   */
/*                                                                          */
/* A pixel p can blend point i only inside the ellipse E: q(p) <= 2 ln(255 o)*/
/* with q(p) = (p - mu)^T Sigma'^-1 (p - mu).  With the option on, E is     */
/* enlarged to q <= tau, tau an upper bound of 2 ln(255 o_max) (o_max: the  */
/* largest opacity any level uses):                                         */
/*   255 o = m 2^e, m in [1, 2):  ln(255 o) = e ln 2 + ln m                 */
/*                                           <= e ln2_up + (m - 1)          */
/* (ln m <= m - 1; ln2_up = the nearest float to ln 2, which lies above it),*/
/* then a relative and an absolute slack of 2^-10.  A tile of the 3-sigma   */
/* rectangle is kept only if the rectangle spanned by its pixel centres,    */
/* [xB+0.5, xB+B-0.5] x [yB+0.5, yB+B-0.5], meets E.  Per tile row this is  */
/* one interval of columns: the strip cuts E in a convex set whose x-shadow */
/* [xl, xr] ends at E's leftmost / rightmost point if that point lies in    */
/* the strip, else where the nearer strip edge dy crosses E,                */
/*   dx = (b dy +- sqrt(det (c tau - dy^2))) / c,                            */
/* with Sigma' = [[a, b], [b, c]], det = a c - b^2, E's x-extent sqrt(tau a)*/
/* reached at dy = b sqrt(tau a) / a, y-extent sqrt(tau c) (the divisions   */
/* taken as products with the rounded reciprocals 1/a, 1/c).  The image is  */
/* unchanged (a dropped tile holds no pixel that could blend the point);    */
/* the tile lists get shorter.  FP32, fixed order, no contraction.          */
/* ------------------------------------------------------------------------ */
#define ORC_SUPP 6   /* u, v, a, b, c, tau */

static float tight_tau(float o) {
  float x = 255.0f * o;
  if (!(x > 1.0f)) return -1.0f;      /* alpha < 1/255 at every pixel */
  int e;
  float m = frexpf(x, &e);            /* x = m 2^e, m in [0.5, 1), exact */
  m = m * 2.0f;
  e = e - 1;
  float t = (float)e * 0.693147182f;
  t = t + (m - 1.0f);
  t = t * 2.0f;
  float sl = t * 0.0009765625f;
  t = t + sl;
  t = t + 0.0009765625f;
  return t;
}

static float strip_end(float b, float ic, float det, float ct, float yb, float sgn) {
  float arg = det * (ct - yb * yb);
  arg = fmaxf(arg, 0.0f);
  float r = b * yb + sgn * sqrtf(arg);
  return r * ic;
}

/* Columns [*xa, *xb] of tile row `by` whose pixel centres can meet the
 * support sp (u, v, a, b, c, tau); 0 if none. */
static int row_interval(const float *sp, int by, int tile, int *xa, int *xb) {
  const float u = sp[0], v = sp[1], a = sp[2], b = sp[3], c = sp[4], tau = sp[5];
  if (!(tau >= 0.0f)) return 0;
  float det = a * c - b * b;
  float dy0 = ((float)(by * tile) + 0.5f) - v;
  float dy1 = ((float)(by * tile + tile - 1) + 0.5f) - v;
  float ye = sqrtf(tau * c);
  if (dy1 < -ye || dy0 > ye) return 0;
  float xe = sqrtf(tau * a);
  float ia = 1.0f / a, ic = 1.0f / c;
  float dys = (b * xe) * ia;
  float ct = c * tau;
  float xr, xl;
  if (dys >= dy0 && dys <= dy1) xr = xe;
  else xr = strip_end(b, ic, det, ct, dys > dy1 ? dy1 : dy0, 1.0f);
  float ndys = -dys;
  if (ndys >= dy0 && ndys <= dy1) xl = -xe;
  else xl = strip_end(b, ic, det, ct, ndys > dy1 ? dy1 : dy0, -1.0f);
  float L = u + xl, R = u + xr;
  float invB = 1.0f / (float)tile;
  float fa = ceilf(((L + 0.5f) - (float)tile) * invB);
  float fb = floorf((R - 0.5f) * invB);
  fa = fminf(fmaxf(fa, -1.0f), 65536.0f);
  fb = fminf(fmaxf(fb, -1.0f), 65536.0f);
  *xa = (int)fa;
  *xb = (int)fb;
  return *xa <= *xb;
}

/* 1 if tile (x, y) is in the support (the tile's row interval holds x). */
static int tile_in_support(const float *sp, int x, int y, int tile) {
  int xa, xb;
  if (!row_interval(sp, y, tile, &xa, &xb)) return 0;
  return x >= xa && x <= xb;
}

static int keyed_one(const float *mu, const float *s, const float *q,
                     const orc_cam *c, int tile, int tiles_x, int tiles_y,
                     uint32_t *dbits, int32_t rect[4], float o_max, float *supp) {
  const float *R = c->R;
  /* camera-space mean: ((R0 x + R1 y) + R2 z) + t */
  float px = R[0] * mu[0];
  px = px + R[1] * mu[1];
  px = px + R[2] * mu[2];
  px = px + c->t[0];
  float py = R[3] * mu[0];
  py = py + R[4] * mu[1];
  py = py + R[5] * mu[2];
  py = py + c->t[1];
  float pz = R[6] * mu[0];
  pz = pz + R[7] * mu[1];
  pz = pz + R[8] * mu[2];
  pz = pz + c->t[2];
  if (!(pz > c->znear) || !(pz < c->zfar)) return 0;

  /* unit quaternion (w, x, y, z); zero -> identity */
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
  /* M = Rq diag(s) */
  float M[9];
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) M[3 * j + k] = r[3 * j + k] * s[k];

  /* Jacobian of the perspective map at the (clamped) camera-space mean */
  float W = (float)c->width, H = (float)c->height;
  float limx = 1.3f * ((0.5f * W) / c->fx);
  float limy = 1.3f * ((0.5f * H) / c->fy);
  float tx = px / pz;
  float ty = py / pz;
  float txc = fminf(fmaxf(tx, -limx), limx);
  float tyc = fminf(fmaxf(ty, -limy), limy);
  float xc = txc * pz;
  float yc = tyc * pz;
  float iz = 1.0f / pz;
  float iz2 = iz * iz;
  float j00 = c->fx * iz;
  float j02 = -((c->fx * xc) * iz2);
  float j11 = c->fy * iz;
  float j12 = -((c->fy * yc) * iz2);
  /* T = J W (2x3) */
  float T0[3], T1[3];
  for (int k = 0; k < 3; ++k) {
    T0[k] = j00 * R[k] + j02 * R[6 + k];
    T1[k] = j11 * R[3 + k] + j12 * R[6 + k];
  }
  /* G = T M (2x3) */
  float G0[3], G1[3];
  for (int k = 0; k < 3; ++k) {
    float g0 = T0[0] * M[k];
    g0 = g0 + T0[1] * M[3 + k];
    g0 = g0 + T0[2] * M[6 + k];
    G0[k] = g0;
    float g1 = T1[0] * M[k];
    g1 = g1 + T1[1] * M[3 + k];
    g1 = g1 + T1[2] * M[6 + k];
    G1[k] = g1;
  }
  /* 2D covariance G G^T + 0.3 I */
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
  if (!(det > 0.0f)) return 0;
  float mid = 0.5f * (a + cc);
  float disc = mid * mid - det;
  disc = fmaxf(0.1f, disc);
  float lam = mid + sqrtf(disc);
  float rad = ceilf(3.0f * sqrtf(lam));
  /* 2D mean */
  float u = c->fx * tx + c->cx;
  float v = c->fy * ty + c->cy;
  /* tile rectangle, inclusive, clamped to the grid */
  float invB = 1.0f / (float)tile;
  float x0 = floorf((u - rad) * invB);
  float x1 = floorf((u + rad) * invB);
  float y0 = floorf((v - rad) * invB);
  float y1 = floorf((v + rad) * invB);
  x0 = fmaxf(x0, 0.0f);
  y0 = fmaxf(y0, 0.0f);
  x1 = fminf(x1, (float)(tiles_x - 1));
  y1 = fminf(y1, (float)(tiles_y - 1));
  if (!(x0 <= x1) || !(y0 <= y1)) return 0;
  rect[0] = (int32_t)x0;
  rect[1] = (int32_t)x1;
  rect[2] = (int32_t)y0;
  rect[3] = (int32_t)y1;
  *dbits = f32_bits(pz);
  if (supp) {
    supp[0] = u;
    supp[1] = v;
    supp[2] = a;
    supp[3] = b;
    supp[4] = cc;
    supp[5] = tight_tau(o_max);
  }
  return 1;
}

int orc_keyed_project(int n, const float *means, const float *scales,
                      const float *quats, const float *opac, const float *sh,
                      int sh_degree, int V, const orc_cam *cams, int tile,
                      const orc_fov *fov, uint8_t *vis, uint32_t *depth_bits,
                      int32_t *rect, float *supp) {
  int S = (sh_degree + 1) * (sh_degree + 1);
  for (int v = 0; v < V; ++v) {
    int tx, ty;
    view_tiles(&cams[v], tile, &tx, &ty);
    /* items are independent: the all-core build (-fopenmp) splits them */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
      int64_t it = (int64_t)v * n + i;
      int fin = 1;
      for (int k = 0; k < 3; ++k)
        fin &= isfinite(means[3 * i + k]) && isfinite(scales[3 * i + k]);
      for (int k = 0; k < 4; ++k) fin &= isfinite(quats[4 * i + k]) != 0;
      fin &= isfinite(opac[i]) != 0;
      for (int k = 0; k < 3 * S; ++k) fin &= isfinite(sh[(int64_t)3 * S * i + k]) != 0;
      depth_bits[it] = 0;
      rect[4 * it] = 0; rect[4 * it + 1] = -1; rect[4 * it + 2] = 0; rect[4 * it + 3] = -1;
      if (!fin) { vis[it] = 2; continue; }
      /* largest opacity any level composites the point with */
      float o_max = opac[i];
      if (fov && fov->opacity_lv)
        for (int l = 0; l < fov->n_levels - 1; ++l)
          o_max = fmaxf(o_max, (float)fov->opacity_lv[(int64_t)l * n + i]);
      vis[it] = (uint8_t)keyed_one(&means[3 * i], &scales[3 * i], &quats[4 * i],
                                   &cams[v], tile, tx, ty, &depth_bits[it],
                                   &rect[4 * it], o_max,
                                   supp ? &supp[ORC_SUPP * it] : NULL);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* foveation levels (keyed FP32)                                            */
/*                                                                          */
/* Sec. 4.1: regions by eccentricity around the gaze, each rendered by its  */
/* level; a better level renders slightly beyond its boundary and the two   */
/* colours are interpolated there.  Readings: ring radius R_k = fy tan(th_k)*/
/* in pixels; level(p) = 1 + #{k : |p-g|^2 >= R_k^2}; the band of boundary k */
/* is R_k <= |p-g| < R_k + band, inside which level k is also needed.       */
/* ------------------------------------------------------------------------ */
typedef struct {
  int level;    /* the pixel's own level (accumulator A) */
  int in_band;  /* 1 if level-1 is also needed (accumulator B) */
  double w;     /* weight of accumulator A; B gets 1 - w */
} fov_px;

static fov_px pixel_level(const orc_cam *c, const orc_fov *fov, int v, int x,
                          int y) {
  fov_px r = {1, 0, 1.0};
  if (!fov || fov->n_levels <= 1) return r;
  if (fov->view_fov && !fov->view_fov[v]) return r;
  float gx = fov->gaze[2 * v], gy = fov->gaze[2 * v + 1];
  float dx = ((float)x + 0.5f) - gx;
  float dy = ((float)y + 0.5f) - gy;
  float d2 = dx * dx + dy * dy;
  int L = fov->n_levels;
  int lvl = 1;
  for (int k = 0; k < L - 1; ++k) {
    float Rk = c->fy * fov->ring_tan[k];
    if (d2 >= Rk * Rk) lvl++;
  }
  r.level = lvl;
  if (lvl >= 2 && fov->band_px > 0.0f) {
    float Rk = c->fy * fov->ring_tan[lvl - 2];
    float Rb = Rk + fov->band_px;
    if (d2 < Rb * Rb) {
      r.in_band = 1;
      double d = sqrt((double)(((double)x + 0.5) - (double)gx) * (((double)x + 0.5) - (double)gx) +
                      (((double)y + 0.5) - (double)gy) * (((double)y + 0.5) - (double)gy));
      double Rd = (double)c->fy * (double)fov->ring_tan[lvl - 2];
      double w = (d - Rd) / (double)fov->band_px;
      if (w < 0.0) w = 0.0;
      if (w > 1.0) w = 1.0;
      r.w = w;
    }
  }
  return r;
}

int orc_tile_levels(int V, const orc_cam *cams, int tile, const orc_fov *fov,
                    uint8_t *tile_level) {
  int64_t base = 0;
  for (int v = 0; v < V; ++v) {
    const orc_cam *c = &cams[v];
    int tx, ty;
    view_tiles(c, tile, &tx, &ty);
    for (int by = 0; by < ty; ++by)
      for (int bx = 0; bx < tx; ++bx) {
        int best = 255;
        for (int y = by * tile; y < (by + 1) * tile && y < c->height; ++y)
          for (int x = bx * tile; x < (bx + 1) * tile && x < c->width; ++x) {
            fov_px p = pixel_level(c, fov, v, x, y);
            int need = p.level - p.in_band;
            if (need < best) best = need;
          }
        tile_level[base + (int64_t)by * tx + bx] = (uint8_t)best;
      }
    base += (int64_t)tx * ty;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* binning: count, emit, stable sort by (tile, depth), ranges               */
/* ------------------------------------------------------------------------ */
static int kept(const uint8_t *tile_level, const uint8_t *bound_m, int64_t gt,
                int i) {
  if (!tile_level || !bound_m) return 1;
  /* Sec. 4.2 filtering: the point takes part in a tile of level t only if
   * t <= m (its quality bound).  With a separate model per level the same
   * rule is conservative: a pixel of level l uses the model of level l (and
   * l - 1 inside a band), never below the tile's level t. */
  return tile_level[gt] <= bound_m[i];
}

int64_t orc_count_pairs(int n, int V, const orc_cam *cams, int tile,
                        const uint8_t *vis, const int32_t *rect,
                        const uint8_t *tile_level, const uint8_t *bound_m,
                        const float *supp, uint32_t *counts) {
  int64_t K = 0;
  for (int v = 0; v < V; ++v) {
    int tx, ty;
    view_tiles(&cams[v], tile, &tx, &ty);
    int64_t tb = tile_base(V, cams, tile, v);
    for (int i = 0; i < n; ++i) {
      int64_t it = (int64_t)v * n + i;
      uint32_t cnt = 0;
      if (vis[it] == 1) {
        const int32_t *rc = &rect[4 * it];
        for (int y = rc[2]; y <= rc[3]; ++y)
          for (int x = rc[0]; x <= rc[1]; ++x)
            cnt += (uint32_t)(kept(tile_level, bound_m, tb + (int64_t)y * tx + x, i) &&
                              (!supp || tile_in_support(&supp[ORC_SUPP * it], x, y, tile)));
      }
      if (counts) counts[it] = cnt;
      K += cnt;
    }
  }
  return K;
}

typedef struct {
  uint64_t key;
  uint32_t val;
  int64_t seq;
} pair_t;

static int cmp_pair(const void *pa, const void *pb) {
  const pair_t *a = (const pair_t *)pa, *b = (const pair_t *)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  /* stability: fall back to emission order */
  return a->seq < b->seq ? -1 : (a->seq > b->seq ? 1 : 0);
}

int orc_bin(int n, int V, const orc_cam *cams, int tile, const uint8_t *vis,
            const uint32_t *depth_bits, const int32_t *rect,
            const uint8_t *tile_level, const uint8_t *bound_m, const float *supp,
            int64_t K, uint64_t *keys, uint32_t *vals, uint32_t *ranges) {
  pair_t *p = (pair_t *)malloc(sizeof(pair_t) * (size_t)(K > 0 ? K : 1));
  if (!p) return -1;
  int64_t k = 0;
  for (int v = 0; v < V; ++v) {
    int tx, ty;
    view_tiles(&cams[v], tile, &tx, &ty);
    int64_t tb = tile_base(V, cams, tile, v);
    for (int i = 0; i < n; ++i) {
      int64_t it = (int64_t)v * n + i;
      if (vis[it] != 1) continue;
      const int32_t *rc = &rect[4 * it];
      for (int y = rc[2]; y <= rc[3]; ++y)
        for (int x = rc[0]; x <= rc[1]; ++x) {
          int64_t gt = tb + (int64_t)y * tx + x;
          if (!kept(tile_level, bound_m, gt, i)) continue;
          if (supp && !tile_in_support(&supp[ORC_SUPP * it], x, y, tile)) continue;
          if (k >= K) { free(p); return -2; }
          p[k].key = ((uint64_t)gt << 32) | depth_bits[it];
          p[k].val = (uint32_t)it;
          p[k].seq = k;
          ++k;
        }
    }
  }
  if (k != K) { free(p); return -3; }
  qsort(p, (size_t)K, sizeof(pair_t), cmp_pair);
  int64_t T = orc_total_tiles(V, cams, tile);
  for (int64_t t = 0; t < T; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
  for (int64_t j = 0; j < K; ++j) {
    keys[j] = p[j].key;
    vals[j] = p[j].val;
    uint64_t t = p[j].key >> 32;
    if (j == 0 || (keys[j - 1] >> 32) != t) ranges[2 * t] = (uint32_t)j;
    ranges[2 * t + 1] = (uint32_t)(j + 1);
  }
  free(p);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* FP64 value projection                                                    */
/* ------------------------------------------------------------------------ */
void orc_sh_basis(const double d[3], double Y[16]) {
  /* Real spherical harmonics, degree <= 3, ordered m = -l..l within each l,
   * equal to sqrt(2) Re Y_l^m (m > 0), sqrt(2) Im Y_l^|m| (m < 0) and Y_l^0
   * of the complex harmonics with the Condon-Shortley phase.  Written as
   * homogeneous polynomials of the unit direction (x, y, z). */
  const double x = d[0], y = d[1], z = d[2];
  const double PI = 3.14159265358979323846;
  const double k1 = sqrt(3.0 / (4.0 * PI));
  const double k2a = 0.5 * sqrt(15.0 / PI);
  const double k2b = 0.25 * sqrt(5.0 / PI);
  const double k2c = 0.25 * sqrt(15.0 / PI);
  const double k3a = 0.25 * sqrt(35.0 / (2.0 * PI));
  const double k3b = 0.5 * sqrt(105.0 / PI);
  const double k3c = 0.25 * sqrt(21.0 / (2.0 * PI));
  const double k3d = 0.25 * sqrt(7.0 / PI);
  const double k3e = 0.25 * sqrt(105.0 / PI);
  const double xx = x * x, yy = y * y, zz = z * z;
  Y[0] = 0.5 / sqrt(PI);
  Y[1] = -k1 * y;
  Y[2] = k1 * z;
  Y[3] = -k1 * x;
  Y[4] = k2a * x * y;
  Y[5] = -k2a * y * z;
  Y[6] = k2b * (2.0 * zz - xx - yy);
  Y[7] = -k2a * x * z;
  Y[8] = k2c * (xx - yy);
  Y[9] = -k3a * y * (3.0 * xx - yy);
  Y[10] = k3b * x * y * z;
  Y[11] = -k3c * y * (4.0 * zz - xx - yy);
  Y[12] = k3d * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
  Y[13] = -k3c * x * (4.0 * zz - xx - yy);
  Y[14] = k3e * z * (xx - yy);
  Y[15] = -k3a * x * (xx - 3.0 * yy);
}

/* Gradient of each basis polynomial with respect to (x, y, z), treating the
 * coordinates as independent (chained through the normalisation later). */
static void sh_basis_grad(const double d[3], double dY[16][3]) {
  const double x = d[0], y = d[1], z = d[2];
  const double PI = 3.14159265358979323846;
  const double k1 = sqrt(3.0 / (4.0 * PI));
  const double k2a = 0.5 * sqrt(15.0 / PI);
  const double k2b = 0.25 * sqrt(5.0 / PI);
  const double k2c = 0.25 * sqrt(15.0 / PI);
  const double k3a = 0.25 * sqrt(35.0 / (2.0 * PI));
  const double k3b = 0.5 * sqrt(105.0 / PI);
  const double k3c = 0.25 * sqrt(21.0 / (2.0 * PI));
  const double k3d = 0.25 * sqrt(7.0 / PI);
  const double k3e = 0.25 * sqrt(105.0 / PI);
  const double xx = x * x, yy = y * y, zz = z * z;
  memset(dY, 0, sizeof(double) * 48);
  dY[1][1] = -k1;
  dY[2][2] = k1;
  dY[3][0] = -k1;
  dY[4][0] = k2a * y;  dY[4][1] = k2a * x;
  dY[5][1] = -k2a * z; dY[5][2] = -k2a * y;
  dY[6][0] = -2.0 * k2b * x; dY[6][1] = -2.0 * k2b * y; dY[6][2] = 4.0 * k2b * z;
  dY[7][0] = -k2a * z; dY[7][2] = -k2a * x;
  dY[8][0] = 2.0 * k2c * x; dY[8][1] = -2.0 * k2c * y;
  /* Y9 = -k3a (3 x^2 y - y^3) */
  dY[9][0] = -k3a * 6.0 * x * y;
  dY[9][1] = -k3a * (3.0 * xx - 3.0 * yy);
  /* Y10 = k3b x y z */
  dY[10][0] = k3b * y * z; dY[10][1] = k3b * x * z; dY[10][2] = k3b * x * y;
  /* Y11 = -k3c (4 y z^2 - x^2 y - y^3) */
  dY[11][0] = -k3c * (-2.0 * x * y);
  dY[11][1] = -k3c * (4.0 * zz - xx - 3.0 * yy);
  dY[11][2] = -k3c * (8.0 * y * z);
  /* Y12 = k3d (2 z^3 - 3 x^2 z - 3 y^2 z) */
  dY[12][0] = k3d * (-6.0 * x * z);
  dY[12][1] = k3d * (-6.0 * y * z);
  dY[12][2] = k3d * (6.0 * zz - 3.0 * xx - 3.0 * yy);
  /* Y13 = -k3c (4 x z^2 - x^3 - x y^2) */
  dY[13][0] = -k3c * (4.0 * zz - 3.0 * xx - yy);
  dY[13][1] = -k3c * (-2.0 * x * y);
  dY[13][2] = -k3c * (8.0 * x * z);
  /* Y14 = k3e (x^2 z - y^2 z) */
  dY[14][0] = k3e * 2.0 * x * z;
  dY[14][1] = -k3e * 2.0 * y * z;
  dY[14][2] = k3e * (xx - yy);
  /* Y15 = -k3a (x^3 - 3 x y^2) */
  dY[15][0] = -k3a * (3.0 * xx - 3.0 * yy);
  dY[15][1] = -k3a * (-6.0 * x * y);
}

/* The basis polynomials and their gradients with every monomial in absolute
 * value (test bookkeeping: the magnitude of the terms behind a gradient,
 * see orc_grad_mag). */
static void sh_basis_abs(const double d[3], double Y[16]) {
  const double x = fabs(d[0]), y = fabs(d[1]), z = fabs(d[2]);
  const double PI = 3.14159265358979323846;
  const double k1 = sqrt(3.0 / (4.0 * PI));
  const double k2a = 0.5 * sqrt(15.0 / PI);
  const double k2b = 0.25 * sqrt(5.0 / PI);
  const double k2c = 0.25 * sqrt(15.0 / PI);
  const double k3a = 0.25 * sqrt(35.0 / (2.0 * PI));
  const double k3b = 0.5 * sqrt(105.0 / PI);
  const double k3c = 0.25 * sqrt(21.0 / (2.0 * PI));
  const double k3d = 0.25 * sqrt(7.0 / PI);
  const double k3e = 0.25 * sqrt(105.0 / PI);
  const double xx = x * x, yy = y * y, zz = z * z;
  Y[0] = 0.5 / sqrt(PI);
  Y[1] = +k1 * y;
  Y[2] = k1 * z;
  Y[3] = +k1 * x;
  Y[4] = k2a * x * y;
  Y[5] = +k2a * y * z;
  Y[6] = k2b * (2.0 * zz + xx + yy);
  Y[7] = +k2a * x * z;
  Y[8] = k2c * (xx + yy);
  Y[9] = +k3a * y * (3.0 * xx + yy);
  Y[10] = k3b * x * y * z;
  Y[11] = +k3c * y * (4.0 * zz + xx + yy);
  Y[12] = k3d * z * (2.0 * zz + 3.0 * xx + 3.0 * yy);
  Y[13] = +k3c * x * (4.0 * zz + xx + yy);
  Y[14] = k3e * z * (xx + yy);
  Y[15] = +k3a * x * (xx + 3.0 * yy);
}

static void sh_basis_grad_abs(const double d[3], double dY[16][3]) {
  const double x = fabs(d[0]), y = fabs(d[1]), z = fabs(d[2]);
  const double PI = 3.14159265358979323846;
  const double k1 = sqrt(3.0 / (4.0 * PI));
  const double k2a = 0.5 * sqrt(15.0 / PI);
  const double k2b = 0.25 * sqrt(5.0 / PI);
  const double k2c = 0.25 * sqrt(15.0 / PI);
  const double k3a = 0.25 * sqrt(35.0 / (2.0 * PI));
  const double k3b = 0.5 * sqrt(105.0 / PI);
  const double k3c = 0.25 * sqrt(21.0 / (2.0 * PI));
  const double k3d = 0.25 * sqrt(7.0 / PI);
  const double k3e = 0.25 * sqrt(105.0 / PI);
  const double xx = x * x, yy = y * y, zz = z * z;
  memset(dY, 0, sizeof(double) * 48);
  dY[1][1] = +k1;
  dY[2][2] = k1;
  dY[3][0] = +k1;
  dY[4][0] = k2a * y;  dY[4][1] = k2a * x;
  dY[5][1] = +k2a * z; dY[5][2] = +k2a * y;
  dY[6][0] = +2.0 * k2b * x; dY[6][1] = +2.0 * k2b * y; dY[6][2] = 4.0 * k2b * z;
  dY[7][0] = +k2a * z; dY[7][2] = +k2a * x;
  dY[8][0] = 2.0 * k2c * x; dY[8][1] = +2.0 * k2c * y;
  dY[9][0] = +k3a * 6.0 * x * y;
  dY[9][1] = +k3a * (3.0 * xx + 3.0 * yy);
  dY[10][0] = k3b * y * z; dY[10][1] = k3b * x * z; dY[10][2] = k3b * x * y;
  dY[11][0] = +k3c * (+2.0 * x * y);
  dY[11][1] = +k3c * (4.0 * zz + xx + 3.0 * yy);
  dY[11][2] = +k3c * (8.0 * y * z);
  dY[12][0] = k3d * (+6.0 * x * z);
  dY[12][1] = k3d * (+6.0 * y * z);
  dY[12][2] = k3d * (6.0 * zz + 3.0 * xx + 3.0 * yy);
  dY[13][0] = +k3c * (4.0 * zz + 3.0 * xx + yy);
  dY[13][1] = +k3c * (+2.0 * x * y);
  dY[13][2] = +k3c * (8.0 * x * z);
  dY[14][0] = k3e * 2.0 * x * z;
  dY[14][1] = +k3e * 2.0 * y * z;
  dY[14][2] = k3e * (xx + yy);
  dY[15][0] = +k3a * (3.0 * xx + 3.0 * yy);
  dY[15][1] = +k3a * (+6.0 * x * y);
}

static void quat_rot(const double *q, double r[9], double qn[4], double *qnorm) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double n = sqrt(w * w + x * x + y * y + z * z);
  *qnorm = n;
  if (n > 0.0) { w /= n; x /= n; y /= n; z /= n; }
  else { w = 1.0; x = y = z = 0.0; }
  qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z;
  r[0] = 1.0 - 2.0 * (y * y + z * z);
  r[1] = 2.0 * (x * y - w * z);
  r[2] = 2.0 * (x * z + w * y);
  r[3] = 2.0 * (x * y + w * z);
  r[4] = 1.0 - 2.0 * (x * x + z * z);
  r[5] = 2.0 * (y * z - w * x);
  r[6] = 2.0 * (x * z - w * y);
  r[7] = 2.0 * (y * z + w * x);
  r[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* Everything the forward and backward need for one (view, point) item. */
typedef struct {
  double pc[3];        /* camera-space mean */
  double xcl, ycl;     /* clamped x, y used by J */
  int clx, cly;        /* clamp active (+1/-1) or 0 */
  double limx, limy;
  double r[9], qn[4], qnorm;
  double M[9];         /* Rq diag(s) */
  double Sig[9];       /* 3D covariance */
  double J[6];         /* 2x3 */
  double T[6];         /* J W */
  double S2[3];        /* 2D covariance a, b, c (with low-pass) */
  double conic[3];
  double u, v;
  double dir[3], dist; /* normalised view direction, distance to camera */
  double Y[16];
  double rgb_raw[3], rgb[3], rest[3];
} item_t;

static void cam_center(const orc_cam *c, double cc[3]) {
  for (int k = 0; k < 3; ++k)
    cc[k] = -((double)c->R[k] * c->t[0] + (double)c->R[3 + k] * c->t[1] +
              (double)c->R[6 + k] * c->t[2]);
}

static void project_item(const double *mu, const double *s, const double *q,
                         const double *sh, int S, const orc_cam *c,
                         item_t *it) {
  double R[9];
  for (int k = 0; k < 9; ++k) R[k] = c->R[k];
  for (int j = 0; j < 3; ++j)
    it->pc[j] = R[3 * j] * mu[0] + R[3 * j + 1] * mu[1] + R[3 * j + 2] * mu[2] + c->t[j];
  double x = it->pc[0], y = it->pc[1], z = it->pc[2];
  quat_rot(q, it->r, it->qn, &it->qnorm);
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) it->M[3 * j + k] = it->r[3 * j + k] * s[k];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += it->M[3 * a + k] * it->M[3 * b + k];
      it->Sig[3 * a + b] = acc;
    }
  double fx = c->fx, fy = c->fy;
  it->limx = CLAMP_FOV * (0.5 * (double)c->width / fx);
  it->limy = CLAMP_FOV * (0.5 * (double)c->height / fy);
  double tx = x / z, ty = y / z;
  it->clx = tx > it->limx ? 1 : (tx < -it->limx ? -1 : 0);
  it->cly = ty > it->limy ? 1 : (ty < -it->limy ? -1 : 0);
  double txc = it->clx ? it->clx * it->limx : tx;
  double tyc = it->cly ? it->cly * it->limy : ty;
  it->xcl = txc * z;
  it->ycl = tyc * z;
  it->J[0] = fx / z; it->J[1] = 0.0; it->J[2] = -fx * it->xcl / (z * z);
  it->J[3] = 0.0; it->J[4] = fy / z; it->J[5] = -fy * it->ycl / (z * z);
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 3; ++k) {
      double acc = 0.0;
      for (int j = 0; j < 3; ++j) acc += it->J[3 * a + j] * R[3 * j + k];
      it->T[3 * a + k] = acc;
    }
  double P[6]; /* T Sigma */
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 3; ++k) {
      double acc = 0.0;
      for (int j = 0; j < 3; ++j) acc += it->T[3 * a + j] * it->Sig[3 * j + k];
      P[3 * a + k] = acc;
    }
  double s00 = 0, s01 = 0, s11 = 0;
  for (int k = 0; k < 3; ++k) {
    s00 += P[k] * it->T[k];
    s01 += P[k] * it->T[3 + k];
    s11 += P[3 + k] * it->T[3 + k];
  }
  it->S2[0] = s00 + LOWPASS;
  it->S2[1] = s01;
  it->S2[2] = s11 + LOWPASS;
  double det = it->S2[0] * it->S2[2] - it->S2[1] * it->S2[1];
  it->conic[0] = it->S2[2] / det;
  it->conic[1] = -it->S2[1] / det;
  it->conic[2] = it->S2[0] / det;
  it->u = fx * x / z + c->cx;
  it->v = fy * y / z + c->cy;
  /* colour: g(SH) at the direction from the camera centre to the mean */
  double cc[3], dv[3];
  cam_center(c, cc);
  for (int k = 0; k < 3; ++k) dv[k] = mu[k] - cc[k];
  it->dist = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  for (int k = 0; k < 3; ++k) it->dir[k] = dv[k] / it->dist;
  orc_sh_basis(it->dir, it->Y);
  for (int ch = 0; ch < 3; ++ch) {
    double rest = 0.0;
    for (int k = 1; k < S; ++k) rest += sh[3 * k + ch] * it->Y[k];
    it->rest[ch] = rest;
    it->rgb_raw[ch] = sh[ch] * it->Y[0] + rest + SH_OFFSET;
    it->rgb[ch] = it->rgb_raw[ch] > 0.0 ? it->rgb_raw[ch] : 0.0;
  }
}

int orc_project_values(int n, const double *means, const double *scales,
                       const double *quats, const double *sh, int sh_degree,
                       int V, const orc_cam *cams, const uint8_t *vis,
                       double *out) {
  int S = (sh_degree + 1) * (sh_degree + 1);
  for (int v = 0; v < V; ++v)
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
      int64_t id = (int64_t)v * n + i;
      double *o = &out[id * ORC_NVAL];
      if (vis[id] != 1) {
        for (int k = 0; k < ORC_NVAL; ++k) o[k] = 0.0;
        continue;
      }
      item_t it;
      project_item(&means[3 * i], &scales[3 * i], &quats[4 * i],
                   &sh[(int64_t)3 * S * i], S, &cams[v], &it);
      o[ORC_U] = it.u; o[ORC_V] = it.v;
      o[ORC_CA] = it.conic[0]; o[ORC_CB] = it.conic[1]; o[ORC_CC] = it.conic[2];
      o[ORC_R] = it.rgb[0]; o[ORC_G] = it.rgb[1]; o[ORC_B] = it.rgb[2];
      o[ORC_RR] = it.rest[0]; o[ORC_RG] = it.rest[1]; o[ORC_RB] = it.rest[2];
      o[ORC_DEPTH] = it.pc[2];
      o[ORC_SA] = it.S2[0]; o[ORC_SB] = it.S2[1]; o[ORC_SC] = it.S2[2];
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* compositing (Eq. 1a)                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
  double C[3], T;
  int32_t last;     /* list position of the last blended point, -1 if none */
  double margin;
  int amb;          /* some decision lies inside its uncertainty window */
  double amb_floor; /* sum of T over ambiguous alpha-floor decisions */
  double amb_stop;  /* T at an ambiguous stop decision (0 if none) */
  double cmax;      /* largest colour channel of the points taking part */
  int64_t dom_item; /* item with the largest T alpha (first maximum) */
  double dom_w;
} acc_t;

/* opacity and colour of item `id` (point i) at level `lvl` */
static double level_opacity(const orc_fov *fov, const double *opac, int n,
                            int i, int lvl) {
  if (lvl >= 2 && fov && fov->opacity_lv)
    return fov->opacity_lv[(int64_t)(lvl - 2) * n + i];
  return opac[i];
}

static void level_colour(const orc_fov *fov, const double *pv, int n, int i,
                         int lvl, double col[3], int clampmask[3]) {
  for (int ch = 0; ch < 3; ++ch) {
    double raw;
    if (lvl >= 2 && fov && fov->dc_lv) {
      raw = pv[ORC_RR + ch] + Y00 * fov->dc_lv[((int64_t)(lvl - 2) * n + i) * 3 + ch] + SH_OFFSET;
      col[ch] = raw > 0.0 ? raw : 0.0;
    } else {
      col[ch] = pv[ORC_R + ch];
      raw = col[ch] > 0.0 ? 1.0 : 0.0;  /* clamp state of the base colour */
    }
    if (clampmask) clampmask[ch] = !(raw > 0.0);
  }
}

static double rel_margin(double a, double thr) {
  return fabs(a / thr - 1.0);
}

/* Decision ambiguity (test bookkeeping, not part of Eq. 1).  The GPU takes
 * the alpha-floor and stop decisions in FP32; near a threshold it may take
 * the other branch.  Error model of its FP32 evaluation:
 *   alpha: log2(alpha) = log2(o) - |t|^2 with t the whitened offset of the
 *     pixel (|t|^2 <= 8 at the floor).  Rounding of t (FMAs over tile-local
 *     coordinates <= 16 px, whitening rows of relative error ~1e-6) and of
 *     log2(o) bound the absolute error of log2(alpha) by ~5e-5, i.e. a
 *     relative error of alpha below ALPHA_REL_ERR = 4e-5; ex2.approx adds
 *     ~2e-7.
 *   T: each blend multiplies by (1 - alpha) rounded twice, so T's relative
 *     error grows per blend by 2 u + ALPHA_REL_ERR alpha / (1 - alpha)
 *     (u = 2^-24; a clamped alpha is 0.99 in FP32, 1e-6 off in 1 - alpha).
 * An alpha-floor decision is ambiguous when alpha lies within AMB_FLOOR
 * (relative) of 1/255; a stop decision when T (1 - alpha) lies within
 * AMB_FLOOR + AMB_SAFE times T's error bound of 1e-4 (the bound adds the
 * per-blend worst cases linearly, so it needs no further safety factor).  Flipping a floor
 * decision at transmittance T changes the pixel by at most 2 T c_max / 255
 * (the point's own T alpha c plus the factor (1 - alpha) on what follows);
 * flipping the stop decision by at most T c_max (everything from there on).
 * A flipped floor decision moves the later T by alpha, which widens the
 * later stop windows. */
#define ALPHA_REL_ERR 4e-5
#define AMB_FLOOR 1e-4
#define AMB_SAFE 1.0
#define U32 5.9604644775390625e-8

/* Whether point i takes part at level lvl (see orc_fov.disjoint).  Without
 * foveation every point takes part. */
static int takes_part(const orc_fov *fov, int i, int lvl) {
  if (!fov || !fov->bound_m) return 1;
  if (fov->disjoint) return fov->bound_m[i] == lvl;
  return lvl <= 1 || fov->bound_m[i] >= lvl;
}

/* Composite one accumulator of one pixel over list positions [s, e).
 * `px`, `py` are the pixel centre.  Only the points that take part at level
 * lvl are composited (takes_part). */
static void composite(int n, const double *vp, const double *opac,
                      const uint32_t *vals, int64_t s, int64_t e,
                      const orc_fov *fov, int lvl, double px, double py,
                      acc_t *acc) {
  acc->C[0] = acc->C[1] = acc->C[2] = 0.0;
  acc->T = 1.0;
  acc->last = -1;
  acc->margin = INFINITY;
  acc->amb = 0;
  acc->amb_floor = 0.0;
  acc->amb_stop = 0.0;
  acc->cmax = 0.0;
  acc->dom_item = -1;
  acc->dom_w = -1.0;
  double errT = 0.0;  /* bound on the relative error of the FP32 T */
  for (int64_t k = s; k < e; ++k) {
    uint32_t id = vals[k];
    int i = (int)(id % (uint32_t)n);
    if (!takes_part(fov, i, lvl)) continue;
    const double *pv = &vp[(int64_t)id * ORC_NVAL];
    double dx = px - pv[ORC_U], dy = py - pv[ORC_V];
    double power = -0.5 * (pv[ORC_CA] * dx * dx + pv[ORC_CC] * dy * dy) - pv[ORC_CB] * dx * dy;
    double o = level_opacity(fov, opac, n, i, lvl);
    double alpha = o * exp(power);
    int clamped = alpha > ALPHA_MAX;
    /* the 0.99 clamp leaves the colour continuous but decides whether the
     * point's geometry and opacity get a gradient: part of the margin */
    double m = rel_margin(alpha, ALPHA_MAX);
    if (m < acc->margin) acc->margin = m;
    if (clamped) alpha = ALPHA_MAX;
    m = rel_margin(alpha, ALPHA_MIN);
    if (m < acc->margin) acc->margin = m;
    if (m < AMB_FLOOR) {
      acc->amb = 1;
      acc->amb_floor += acc->T;
      errT += alpha; /* the other branch scales the later T by 1 - alpha */
    }
    if (alpha < ALPHA_MIN) continue;
    double Tn = acc->T * (1.0 - alpha);
    errT += 2.0 * U32 + (clamped ? 1e-6 : ALPHA_REL_ERR * alpha / (1.0 - alpha));
    m = rel_margin(Tn, T_MIN);
    if (m < acc->margin) acc->margin = m;
    if (m < AMB_FLOOR + AMB_SAFE * errT) {
      acc->amb = 1;
      if (acc->T > acc->amb_stop) acc->amb_stop = acc->T;
    }
    if (Tn < T_MIN) break;
    double col[3];
    level_colour(fov, pv, n, i, lvl, col, NULL);
    double w = acc->T * alpha;
    if (w > acc->dom_w) { acc->dom_w = w; acc->dom_item = id; }
    for (int ch = 0; ch < 3; ++ch) acc->C[ch] += w * col[ch];
    acc->T = Tn;
    acc->last = (int32_t)(k - s);
  }
  if (acc->amb) {
    /* largest colour any point of the list contributes at this level: bounds
     * what a flipped decision adds or removes */
    for (int64_t k = s; k < e; ++k) {
      uint32_t id = vals[k];
      int i = (int)(id % (uint32_t)n);
      if (!takes_part(fov, i, lvl)) continue;
      double col[3];
      level_colour(fov, &vp[(int64_t)id * ORC_NVAL], n, i, lvl, col, NULL);
      for (int ch = 0; ch < 3; ++ch)
        if (col[ch] > acc->cmax) acc->cmax = col[ch];
    }
  }
}

/* What flipping the ambiguous decisions of an accumulator can change in its
 * colour (see the error model above); bg enters like a colour. */
static double amb_bound(const acc_t *a, const double bg[3]) {
  if (!a->amb) return 0.0;
  double c = a->cmax;
  for (int ch = 0; ch < 3; ++ch)
    if (bg[ch] > c) c = bg[ch];
  return (2.0 * ALPHA_MIN * (1.0 + AMB_FLOOR)) * c * a->amb_floor + c * a->amb_stop;
}

static int find_view(int V, const orc_cam *cams, int64_t gp, int *x, int *y) {
  int64_t b = 0;
  for (int v = 0; v < V; ++v) {
    int64_t np = (int64_t)cams[v].width * cams[v].height;
    if (gp < b + np) {
      int64_t l = gp - b;
      *x = (int)(l % cams[v].width);
      *y = (int)(l / cams[v].width);
      return v;
    }
    b += np;
  }
  return -1;
}

/* Render one pixel from a list [s, e) of items; writes its outputs. */
static void shade_pixel(int n, int V, const orc_cam *cams, const double *vp,
                        const double *opac, const uint32_t *vals, int64_t s,
                        int64_t e, const orc_fov *fov, const double bg[3],
                        int v, int x, int y, double *rgb, double *T,
                        int32_t *last, double *margin, double *wband,
                        double *ambB, uint8_t *amb, acc_t *outA) {
  (void)V;
  fov_px fp = pixel_level(&cams[v], fov, v, x, y);
  double px = x + 0.5, py = y + 0.5;
  acc_t A, B;
  composite(n, vp, opac, vals, s, e, fov, fp.level, px, py, &A);
  double mg = A.margin;
  int am = A.amb;
  double ab = (fp.in_band ? fp.w : 1.0) * amb_bound(&A, bg);
  double out[3];
  for (int ch = 0; ch < 3; ++ch) out[ch] = A.C[ch] + A.T * bg[ch];
  T[0] = A.T; last[0] = A.last;
  T[1] = 1.0; last[1] = -1;
  if (fp.in_band) {
    composite(n, vp, opac, vals, s, e, fov, fp.level - 1, px, py, &B);
    if (B.margin < mg) mg = B.margin;
    am |= B.amb;
    ab += (1.0 - fp.w) * amb_bound(&B, bg);
    for (int ch = 0; ch < 3; ++ch)
      out[ch] = fp.w * out[ch] + (1.0 - fp.w) * (B.C[ch] + B.T * bg[ch]);
    T[1] = B.T; last[1] = B.last;
  }
  for (int ch = 0; ch < 3; ++ch) rgb[ch] = out[ch];
  if (margin) *margin = mg;
  if (wband) *wband = fp.w;
  if (ambB) *ambB = ab;
  if (amb) *amb = (uint8_t)am;
  if (outA) *outA = A;
}

int orc_render(int n, int V, const orc_cam *cams, int tile,
               const double *vp, const double *opac, const uint32_t *vals,
               const uint32_t *ranges, const orc_fov *fov, const double bg[3],
               const int64_t *pix, int64_t npix, double *rgb, double *T,
               int32_t *last, double *margin, double *wband, double *ambB,
               uint8_t *amb, uint32_t *stats) {
  if (pix) {
    int bad = 0;
    /* pixels are independent: the all-core build (-fopenmp) splits them */
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
    for (int64_t q = 0; q < npix; ++q) {
      int x, y;
      int v = find_view(V, cams, pix[q], &x, &y);
      if (v < 0) {
        bad = 1;
        continue;
      }
      int tx, ty;
      view_tiles(&cams[v], tile, &tx, &ty);
      int64_t gt = tile_base(V, cams, tile, v) + (int64_t)(y / tile) * tx + x / tile;
      shade_pixel(n, V, cams, vp, opac, vals, ranges[2 * gt], ranges[2 * gt + 1], fov,
                  bg, v, x, y, &rgb[3 * q], &T[2 * q], &last[2 * q],
                  margin ? &margin[q] : NULL, wband ? &wband[q] : NULL,
                  ambB ? &ambB[q] : NULL, amb ? &amb[q] : NULL, NULL);
    }
    return bad ? -1 : 0;
  }
  /* whole batch, tile by tile (so that per-tile statistics are exact) */
  uint32_t *tt = stats, *tu = stats ? stats + n : NULL, *pb = stats ? stats + 2 * (int64_t)n : NULL,
           *pd = stats ? stats + 3 * (int64_t)n : NULL;
  if (stats) memset(stats, 0, sizeof(uint32_t) * 4 * (size_t)n);
  int64_t maxlen = 0;
  int64_t Ttot = orc_total_tiles(V, cams, tile);
  for (int64_t t = 0; t < Ttot; ++t) {
    int64_t l = (int64_t)ranges[2 * t + 1] - ranges[2 * t];
    if (l > maxlen) maxlen = l;
  }
  uint8_t *used = (uint8_t *)calloc((size_t)(maxlen > 0 ? maxlen : 1), 1);
  int64_t tb = 0;
  for (int v = 0; v < V; ++v) {
    const orc_cam *c = &cams[v];
    int tx, ty;
    view_tiles(c, tile, &tx, &ty);
    int64_t pb0 = pix_base(cams, v);
    for (int by = 0; by < ty; ++by)
      for (int bx = 0; bx < tx; ++bx) {
        int64_t gt = tb + (int64_t)by * tx + bx;
        int64_t s = ranges[2 * gt], e = ranges[2 * gt + 1];
        if (stats) {
          memset(used, 0, (size_t)(e - s > 0 ? e - s : 0));
          for (int64_t k = s; k < e; ++k) tt[vals[k] % (uint32_t)n]++;
        }
        for (int y = by * tile; y < (by + 1) * tile && y < c->height; ++y)
          for (int x = bx * tile; x < (bx + 1) * tile && x < c->width; ++x) {
            int64_t q = pb0 + (int64_t)y * c->width + x;
            acc_t A;
            shade_pixel(n, V, cams, vp, opac, vals, s, e, fov, bg, v, x, y,
                        &rgb[3 * q], &T[2 * q], &last[2 * q],
                        margin ? &margin[q] : NULL, wband ? &wband[q] : NULL,
                        ambB ? &ambB[q] : NULL, amb ? &amb[q] : NULL, &A);
            if (stats && A.last >= 0) {
              /* re-walk to mark blended points (statistics of accumulator A) */
              fov_px fp = pixel_level(c, fov, v, x, y);
              double px = x + 0.5, py = y + 0.5, Tc = 1.0;
              for (int64_t k = s; k <= s + A.last; ++k) {
                uint32_t id = vals[k];
                int i = (int)(id % (uint32_t)n);
                if (!takes_part(fov, i, fp.level)) continue;
                const double *pv = &vp[(int64_t)id * ORC_NVAL];
                double dx = px - pv[ORC_U], dy = py - pv[ORC_V];
                double power = -0.5 * (pv[ORC_CA] * dx * dx + pv[ORC_CC] * dy * dy) - pv[ORC_CB] * dx * dy;
                double alpha = level_opacity(fov, opac, n, i, fp.level) * exp(power);
                if (alpha > ALPHA_MAX) alpha = ALPHA_MAX;
                if (alpha < ALPHA_MIN) continue;
                used[k - s] = 1;
                pb[i]++;
                Tc *= (1.0 - alpha);
              }
              pd[A.dom_item % (uint32_t)n]++;
            }
          }
        if (stats)
          for (int64_t k = s; k < e; ++k)
            if (used[k - s]) tu[vals[k] % (uint32_t)n]++;
      }
    tb += (int64_t)tx * ty;
  }
  free(used);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* brute force (no tile lists)                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t dbits;
  uint32_t id;
} bf_t;

static int cmp_bf(const void *pa, const void *pb) {
  const bf_t *a = (const bf_t *)pa, *b = (const bf_t *)pb;
  if (a->dbits != b->dbits) return a->dbits < b->dbits ? -1 : 1;
  return a->id < b->id ? -1 : (a->id > b->id ? 1 : 0);
}

int orc_render_brute(int n, int V, const orc_cam *cams, int tile,
                     const uint8_t *vis, const uint32_t *depth_bits,
                     const int32_t *rect, const double *vp, const double *opac,
                     const orc_fov *fov, const double bg[3], double *rgb,
                     double *T, int32_t *last) {
  bf_t *lst = (bf_t *)malloc(sizeof(bf_t) * (size_t)(n > 0 ? n : 1));
  uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  if (!lst || !ids) { free(lst); free(ids); return -1; }
  for (int v = 0; v < V; ++v) {
    const orc_cam *c = &cams[v];
    int tx, ty;
    view_tiles(c, tile, &tx, &ty);
    int64_t pb0 = pix_base(cams, v);
    for (int y = 0; y < c->height; ++y)
      for (int x = 0; x < c->width; ++x) {
        int bx = x / tile, by = y / tile;
        int cnt = 0;
        for (int i = 0; i < n; ++i) {
          int64_t id = (int64_t)v * n + i;
          if (vis[id] != 1) continue;
          const int32_t *rc = &rect[4 * id];
          if (bx < rc[0] || bx > rc[1] || by < rc[2] || by > rc[3]) continue;
          lst[cnt].dbits = depth_bits[id];
          lst[cnt].id = (uint32_t)id;
          ++cnt;
        }
        qsort(lst, (size_t)cnt, sizeof(bf_t), cmp_bf);
        for (int k = 0; k < cnt; ++k) ids[k] = lst[k].id;
        int64_t q = pb0 + (int64_t)y * c->width + x;
        shade_pixel(n, V, cams, vp, opac, ids, 0, cnt, fov, bg, v, x, y,
                    &rgb[3 * q], &T[2 * q], &last[2 * q], NULL, NULL, NULL, NULL, NULL);
        /* list positions of this per-pixel list -> items */
        for (int a = 0; a < 2; ++a)
          if (last[2 * q + a] >= 0) last[2 * q + a] = (int32_t)ids[last[2 * q + a]];
      }
  }
  free(lst);
  free(ids);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* analytic FP64 gradient                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  double dmu2[2];   /* dL / d mean2D */
  double dconic[3]; /* dL / d(a, b, c) of the conic [[a, b], [b, c]] */
} g2d_t;

/* Backward through one accumulator of one pixel with upstream g[3]:
 * rebuilds the blended list in order, then applies
 *   dL/dc_i     = T_i alpha_i g
 *   dL/dalpha_i = g . (T_i c_i - (S_i + T_final bg) / (1 - alpha_i)),
 *   S_i = sum_{j > i} T_j alpha_j c_j,
 * then alpha = min(0.99, o exp(power)), power = -1/2 d^T Q d, d = p - mu. */
static void backward_acc(int n, const double *vp, const double *opac,
                         const uint32_t *vals, int64_t s, int64_t e,
                         const orc_fov *fov, int lvl, double px, double py,
                         const double g[3], const double bg[3], g2d_t *g2,
                         double *dop_lv, double *dcol_lv, int L, int64_t nitems,
                         g2d_t *g2a, double *dopa_lv, double *dcola_lv) {
  /* forward pass recording the blended points */
  int64_t cap = e - s > 0 ? e - s : 1;
  int64_t *bk = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
  double *ba = (double *)malloc(sizeof(double) * (size_t)cap);
  double *bT = (double *)malloc(sizeof(double) * (size_t)cap);
  double *bc = (double *)malloc(sizeof(double) * 3 * (size_t)cap);
  int *bcl = (int *)malloc(sizeof(int) * (size_t)cap);
  int nb = 0;
  double T = 1.0;
  for (int64_t k = s; k < e; ++k) {
    uint32_t id = vals[k];
    int i = (int)(id % (uint32_t)n);
    if (!takes_part(fov, i, lvl)) continue;
    const double *pv = &vp[(int64_t)id * ORC_NVAL];
    double dx = px - pv[ORC_U], dy = py - pv[ORC_V];
    double power = -0.5 * (pv[ORC_CA] * dx * dx + pv[ORC_CC] * dy * dy) - pv[ORC_CB] * dx * dy;
    double o = level_opacity(fov, opac, n, i, lvl);
    double a0 = o * exp(power);
    double alpha = a0 > ALPHA_MAX ? ALPHA_MAX : a0;
    if (alpha < ALPHA_MIN) continue;
    double Tn = T * (1.0 - alpha);
    if (Tn < T_MIN) break;
    bk[nb] = k;
    ba[nb] = alpha;
    bT[nb] = T;
    level_colour(fov, pv, n, i, lvl, &bc[3 * nb], NULL);
    bcl[nb] = a0 > ALPHA_MAX;
    ++nb;
    T = Tn;
  }
  double S[3] = {T * bg[0], T * bg[1], T * bg[2]}; /* S_i + T_final bg */
  for (int j = nb - 1; j >= 0; --j) {
    uint32_t id = vals[bk[j]];
    int i = (int)(id % (uint32_t)n);
    const double *pv = &vp[(int64_t)id * ORC_NVAL];
    double a = ba[j], Ti = bT[j];
    double dalpha = 0.0, dalpha_a = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
      double dc = Ti * a * g[ch];
      dcol_lv[((int64_t)(lvl - 1) * nitems + id) * 3 + ch] += dc;
      dalpha += g[ch] * (Ti * bc[3 * j + ch] - S[ch] / (1.0 - a));
      if (g2a) {
        dcola_lv[((int64_t)(lvl - 1) * nitems + id) * 3 + ch] += fabs(dc);
        dalpha_a += fabs(g[ch]) * (Ti * bc[3 * j + ch] + S[ch] / (1.0 - a));
      }
    }
    for (int ch = 0; ch < 3; ++ch) S[ch] += Ti * a * bc[3 * j + ch];
    if (bcl[j]) continue; /* clamped at 0.99: no gradient to o or geometry */
    double o = level_opacity(fov, opac, n, i, lvl);
    double ex = a / o; /* exp(power) */
    dop_lv[(int64_t)(lvl - 1) * nitems + id] += dalpha * ex;
    double dpow = dalpha * a;
    double dx = px - pv[ORC_U], dy = py - pv[ORC_V];
    /* d power / d mu = Q d */
    g2[id].dmu2[0] += dpow * (pv[ORC_CA] * dx + pv[ORC_CB] * dy);
    g2[id].dmu2[1] += dpow * (pv[ORC_CB] * dx + pv[ORC_CC] * dy);
    g2[id].dconic[0] += dpow * (-0.5 * dx * dx);
    g2[id].dconic[1] += dpow * (-dx * dy);
    g2[id].dconic[2] += dpow * (-0.5 * dy * dy);
    if (g2a) {
      /* the same terms in absolute value (test bookkeeping, see orc_grad_mag) */
      double dpa = dalpha_a * a;
      dopa_lv[(int64_t)(lvl - 1) * nitems + id] += dalpha_a * ex;
      g2a[id].dmu2[0] += dpa * (fabs(pv[ORC_CA] * dx) + fabs(pv[ORC_CB] * dy));
      g2a[id].dmu2[1] += dpa * (fabs(pv[ORC_CB] * dx) + fabs(pv[ORC_CC] * dy));
      g2a[id].dconic[0] += dpa * (0.5 * dx * dx);
      g2a[id].dconic[1] += dpa * fabs(dx * dy);
      g2a[id].dconic[2] += dpa * (0.5 * dy * dy);
    }
  }
  (void)L;
  free(bk); free(ba); free(bT); free(bc); free(bcl);
}

/* The chain of one item to its point's parameters with every term in
 * absolute value (test bookkeeping): a bound of the sum of the magnitudes of
 * the terms each gradient element sums, the scale of its rounding error in
 * a finite-precision evaluation.  Inputs: the absolute 2D and per-level
 * sums of the item (ga, dopa, dcola); adds into mag. */
static void chain_item_abs(const item_t *it, const orc_cam *c, const double *shi, int S, int L,
                           const orc_fov *fov, int n, int i, const double *scales,
                           const g2d_t *ga, const double *dopa, const double *dcola,
                           int64_t nitems, int64_t id, const orc_grad_mag *mag) {
  double R[9];
  for (int k = 0; k < 9; ++k) R[k] = fabs((double)c->R[k]);
  double Ya[16];
  sh_basis_abs(it->dir, Ya);
  double dcb[3] = {0, 0, 0};
  for (int l = 1; l <= L; ++l) {
    double dop_l = dopa[(int64_t)(l - 1) * nitems + id];
    const double *dc = &dcola[((int64_t)(l - 1) * nitems + id) * 3];
    if (l >= 2 && fov && fov->opacity_lv) {
      if (mag->opac_lv) mag->opac_lv[(int64_t)(l - 2) * n + i] += dop_l;
    } else if (mag->opac) {
      mag->opac[i] += dop_l;
    }
    if (l >= 2 && fov && fov->dc_lv) {
      for (int ch = 0; ch < 3; ++ch) {
        if (mag->dc_lv) mag->dc_lv[((int64_t)(l - 2) * n + i) * 3 + ch] += Y00 * dc[ch];
        if (mag->sh)
          for (int k = 1; k < S; ++k) mag->sh[(int64_t)3 * S * i + 3 * k + ch] += Ya[k] * dc[ch];
      }
    } else {
      for (int ch = 0; ch < 3; ++ch) dcb[ch] += dc[ch];
    }
  }
  double dY[16];
  for (int k = 0; k < 16; ++k) dY[k] = 0.0;
  for (int ch = 0; ch < 3; ++ch)
    for (int k = 0; k < S; ++k) {
      if (mag->sh) mag->sh[(int64_t)3 * S * i + 3 * k + ch] += Ya[k] * dcb[ch];
      dY[k] += fabs(shi[3 * k + ch]) * dcb[ch];
    }
  if (fov && fov->dc_lv)
    for (int l = 2; l <= L; ++l) {
      const double *dc = &dcola[((int64_t)(l - 1) * nitems + id) * 3];
      for (int ch = 0; ch < 3; ++ch)
        for (int k = 1; k < S; ++k) dY[k] += fabs(shi[3 * k + ch]) * dc[ch];
    }
  double gY[16][3];
  sh_basis_grad_abs(it->dir, gY);
  double ddir[3] = {0, 0, 0};
  for (int k = 1; k < S; ++k)
    for (int a = 0; a < 3; ++a) ddir[a] += dY[k] * gY[k][a];
  double dd = ddir[0] * fabs(it->dir[0]) + ddir[1] * fabs(it->dir[1]) + ddir[2] * fabs(it->dir[2]);
  double dm[3];
  for (int a = 0; a < 3; ++a) dm[a] = (ddir[a] + dd * fabs(it->dir[a])) / it->dist;
  /* conic -> 2D covariance -> T, Sigma -> M -> scales, rotation */
  double Q[4] = {fabs(it->conic[0]), fabs(it->conic[1]), fabs(it->conic[1]), fabs(it->conic[2])};
  double dQ[4] = {ga->dconic[0], 0.5 * ga->dconic[1], 0.5 * ga->dconic[1], ga->dconic[2]};
  double tmp[4], dS2[4];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) tmp[2 * a + b] = dQ[2 * a] * Q[b] + dQ[2 * a + 1] * Q[2 + b];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) dS2[2 * a + b] = Q[2 * a] * tmp[b] + Q[2 * a + 1] * tmp[2 + b];
  double Ta[6], Sa[9], Ma[9], ra[9];
  for (int k = 0; k < 6; ++k) Ta[k] = fabs(it->T[k]);
  for (int k = 0; k < 9; ++k) { Sa[k] = fabs(it->Sig[k]); Ma[k] = fabs(it->M[k]); ra[k] = fabs(it->r[k]); }
  double TS[6];
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 3; ++k) {
      double acc = 0.0;
      for (int j = 0; j < 3; ++j) acc += Ta[3 * a + j] * Sa[3 * j + k];
      TS[3 * a + k] = acc;
    }
  double dT[6];
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 3; ++k) dT[3 * a + k] = 2.0 * (dS2[2 * a] * TS[k] + dS2[2 * a + 1] * TS[3 + k]);
  double dSig[9];
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) {
      double acc = 0.0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) acc += Ta[3 * a + j] * dS2[2 * a + b] * Ta[3 * b + k];
      dSig[3 * j + k] = acc;
    }
  double dM[9];
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) {
      double acc = 0.0;
      for (int l = 0; l < 3; ++l) acc += (dSig[3 * j + l] + dSig[3 * l + j]) * Ma[3 * l + k];
      dM[3 * j + k] = acc;
    }
  const double *s3 = &scales[3 * i];
  double dR[9];
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) {
      if (mag->scales) mag->scales[3 * i + k] += dM[3 * j + k] * ra[3 * j + k];
      dR[3 * j + k] = dM[3 * j + k] * fabs(s3[k]);
    }
  double w = fabs(it->qn[0]), x = fabs(it->qn[1]), y = fabs(it->qn[2]), z = fabs(it->qn[3]);
  double dq[4];
  dq[0] = 2.0 * (z * dR[1] + y * dR[2] + z * dR[3] + x * dR[5] + y * dR[6] + x * dR[7]);
  dq[1] = 2.0 * (y * dR[1] + z * dR[2] + y * dR[3] + 2.0 * x * dR[4] + w * dR[5] + z * dR[6] +
                 w * dR[7] + 2.0 * x * dR[8]);
  dq[2] = 2.0 * (2.0 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] + w * dR[6] +
                 z * dR[7] + 2.0 * y * dR[8]);
  dq[3] = 2.0 * (2.0 * z * dR[0] + w * dR[1] + x * dR[2] + w * dR[3] + 2.0 * z * dR[4] +
                 y * dR[5] + x * dR[6] + y * dR[7]);
  if (it->qnorm > 0.0 && mag->quats) {
    double dot = dq[0] * w + dq[1] * x + dq[2] * y + dq[3] * z;
    mag->quats[4 * i + 0] += (dq[0] + dot * w) / it->qnorm;
    mag->quats[4 * i + 1] += (dq[1] + dot * x) / it->qnorm;
    mag->quats[4 * i + 2] += (dq[2] + dot * y) / it->qnorm;
    mag->quats[4 * i + 3] += (dq[3] + dot * z) / it->qnorm;
  }
  /* T = J W -> J -> camera-space mean; 2D mean -> camera-space mean */
  double dJ[6];
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += dT[3 * a + k] * R[3 * j + k];
      dJ[3 * a + j] = acc;
    }
  double pz = fabs(it->pc[2]), px = fabs(it->pc[0]), py = fabs(it->pc[1]);
  double fx = fabs(c->fx), fy = fabs(c->fy), xcl = fabs(it->xcl), ycl = fabs(it->ycl);
  double dpc[3] = {0, 0, 0};
  dpc[2] += dJ[0] * fx / (pz * pz) + dJ[4] * fy / (pz * pz) + dJ[2] * 2.0 * fx * xcl / (pz * pz * pz) +
            dJ[5] * 2.0 * fy * ycl / (pz * pz * pz);
  double dxcl = dJ[2] * fx / (pz * pz), dycl = dJ[5] * fy / (pz * pz);
  if (it->clx) dpc[2] += dxcl * it->limx; else dpc[0] += dxcl;
  if (it->cly) dpc[2] += dycl * it->limy; else dpc[1] += dycl;
  double du = ga->dmu2[0], dv = ga->dmu2[1];
  dpc[0] += du * fx / pz;
  dpc[1] += dv * fy / pz;
  dpc[2] += du * fx * px / (pz * pz) + dv * fy * py / (pz * pz);
  if (mag->means)
    for (int a = 0; a < 3; ++a)
      mag->means[3 * i + a] += dm[a] + R[a] * dpc[0] + R[3 + a] * dpc[1] + R[6 + a] * dpc[2];
}

int orc_backward(int n, const double *means, const double *scales,
                 const double *quats, const double *opac, const double *sh,
                 int sh_degree, int V, const orc_cam *cams, int tile,
                 const uint32_t *vals, const uint32_t *ranges,
                 const orc_fov *fov, const double bg[3],
                 const double *dL_drgb, double *d_means, double *d_scales,
                 double *d_quats, double *d_opac, double *d_sh,
                 double *d_opac_lv, double *d_dc_lv, const orc_grad_mag *mag) {
  int S = (sh_degree + 1) * (sh_degree + 1);
  int L = (fov && fov->n_levels > 1) ? fov->n_levels : 1;
  int64_t nitems = (int64_t)V * n;
  /* visibility of items follows from the lists: recompute the value record
   * for every item that appears in some list */
  uint8_t *vis = (uint8_t *)calloc((size_t)nitems, 1);
  int64_t Ttot = orc_total_tiles(V, cams, tile);
  for (int64_t t = 0; t < Ttot; ++t)
    for (uint32_t k = ranges[2 * t]; k < ranges[2 * t + 1]; ++k) vis[vals[k]] = 1;
  double *vp = (double *)calloc((size_t)nitems * ORC_NVAL, sizeof(double));
  item_t *items = (item_t *)calloc((size_t)nitems, sizeof(item_t));
  g2d_t *g2 = (g2d_t *)calloc((size_t)nitems, sizeof(g2d_t));
  double *dop = (double *)calloc((size_t)nitems * L, sizeof(double));
  double *dcol = (double *)calloc((size_t)nitems * L * 3, sizeof(double));
  if (!vis || !vp || !items || !g2 || !dop || !dcol) return -1;
  g2d_t *g2a = NULL;
  double *dopa = NULL, *dcola = NULL;
  if (mag) {
    g2a = (g2d_t *)calloc((size_t)nitems, sizeof(g2d_t));
    dopa = (double *)calloc((size_t)nitems * L, sizeof(double));
    dcola = (double *)calloc((size_t)nitems * L * 3, sizeof(double));
    if (!g2a || !dopa || !dcola) return -1;
  }
  for (int v = 0; v < V; ++v)
    for (int i = 0; i < n; ++i) {
      int64_t id = (int64_t)v * n + i;
      if (!vis[id]) continue;
      item_t *it = &items[id];
      project_item(&means[3 * i], &scales[3 * i], &quats[4 * i],
                   &sh[(int64_t)3 * S * i], S, &cams[v], it);
      double *o = &vp[id * ORC_NVAL];
      o[ORC_U] = it->u; o[ORC_V] = it->v;
      o[ORC_CA] = it->conic[0]; o[ORC_CB] = it->conic[1]; o[ORC_CC] = it->conic[2];
      o[ORC_R] = it->rgb[0]; o[ORC_G] = it->rgb[1]; o[ORC_B] = it->rgb[2];
      o[ORC_RR] = it->rest[0]; o[ORC_RG] = it->rest[1]; o[ORC_RB] = it->rest[2];
    }
  /* pixels */
  int64_t tb = 0, pb0 = 0;
  for (int v = 0; v < V; ++v) {
    const orc_cam *c = &cams[v];
    int tx, ty;
    view_tiles(c, tile, &tx, &ty);
    for (int y = 0; y < c->height; ++y)
      for (int x = 0; x < c->width; ++x) {
        int64_t q = pb0 + (int64_t)y * c->width + x;
        int64_t gt = tb + (int64_t)(y / tile) * tx + x / tile;
        int64_t s = ranges[2 * gt], e = ranges[2 * gt + 1];
        fov_px fp = pixel_level(c, fov, v, x, y);
        const double *g = &dL_drgb[3 * q];
        double gA[3], gB[3];
        double wA = fp.in_band ? fp.w : 1.0;
        for (int ch = 0; ch < 3; ++ch) { gA[ch] = wA * g[ch]; gB[ch] = (1.0 - wA) * g[ch]; }
        backward_acc(n, vp, opac, vals, s, e, fov, fp.level, x + 0.5, y + 0.5,
                     gA, bg, g2, dop, dcol, L, nitems, g2a, dopa, dcola);
        if (fp.in_band)
          backward_acc(n, vp, opac, vals, s, e, fov, fp.level - 1, x + 0.5, y + 0.5,
                       gB, bg, g2, dop, dcol, L, nitems, g2a, dopa, dcola);
      }
    tb += (int64_t)tx * ty;
    pb0 += (int64_t)c->width * c->height;
  }
  /* chain each item to the 3D parameters */
  memset(d_means, 0, sizeof(double) * 3 * (size_t)n);
  memset(d_scales, 0, sizeof(double) * 3 * (size_t)n);
  memset(d_quats, 0, sizeof(double) * 4 * (size_t)n);
  memset(d_opac, 0, sizeof(double) * (size_t)n);
  memset(d_sh, 0, sizeof(double) * 3 * (size_t)S * n);
  if (d_opac_lv) memset(d_opac_lv, 0, sizeof(double) * (size_t)(L - 1) * n);
  if (d_dc_lv) memset(d_dc_lv, 0, sizeof(double) * (size_t)(L - 1) * n * 3);
  if (mag) {
    if (mag->means) memset(mag->means, 0, sizeof(double) * 3 * (size_t)n);
    if (mag->scales) memset(mag->scales, 0, sizeof(double) * 3 * (size_t)n);
    if (mag->quats) memset(mag->quats, 0, sizeof(double) * 4 * (size_t)n);
    if (mag->opac) memset(mag->opac, 0, sizeof(double) * (size_t)n);
    if (mag->sh) memset(mag->sh, 0, sizeof(double) * 3 * (size_t)S * n);
    if (mag->opac_lv) memset(mag->opac_lv, 0, sizeof(double) * (size_t)(L - 1) * n);
    if (mag->dc_lv) memset(mag->dc_lv, 0, sizeof(double) * (size_t)(L - 1) * n * 3);
  }
  for (int v = 0; v < V; ++v) {
    const orc_cam *c = &cams[v];
    double R[9];
    for (int k = 0; k < 9; ++k) R[k] = c->R[k];
    for (int i = 0; i < n; ++i) {
      int64_t id = (int64_t)v * n + i;
      if (!vis[id]) continue;
      item_t *it = &items[id];
      const double *shi = &sh[(int64_t)3 * S * i];
      if (mag)
        chain_item_abs(it, c, shi, S, L, fov, n, i, scales, &g2a[id], dopa, dcola, nitems, id, mag);
      /* opacity and colour, per level */
      double dcolor_base[3] = {0, 0, 0};
      for (int l = 1; l <= L; ++l) {
        double dop_l = dop[(int64_t)(l - 1) * nitems + id];
        const double *dc = &dcol[((int64_t)(l - 1) * nitems + id) * 3];
        if (l >= 2 && fov && fov->opacity_lv) d_opac_lv[(int64_t)(l - 2) * n + i] += dop_l;
        else d_opac[i] += dop_l;
        if (l >= 2 && fov && fov->dc_lv) {
          for (int ch = 0; ch < 3; ++ch) {
            double raw = it->rest[ch] + Y00 * fov->dc_lv[((int64_t)(l - 2) * n + i) * 3 + ch] + SH_OFFSET;
            if (!(raw > 0.0)) continue;
            d_dc_lv[((int64_t)(l - 2) * n + i) * 3 + ch] += Y00 * dc[ch];
            /* the view-dependent part is shared with the base colour */
            for (int k = 1; k < S; ++k) d_sh[(int64_t)3 * S * i + 3 * k + ch] += it->Y[k] * dc[ch];
          }
        } else {
          for (int ch = 0; ch < 3; ++ch) dcolor_base[ch] += dc[ch];
        }
      }
      /* SH of the base colour (clamped channels get nothing) */
      double dY[16];
      for (int k = 0; k < 16; ++k) dY[k] = 0.0;
      for (int ch = 0; ch < 3; ++ch) {
        if (!(it->rgb_raw[ch] > 0.0)) continue;
        for (int k = 0; k < S; ++k) {
          d_sh[(int64_t)3 * S * i + 3 * k + ch] += it->Y[k] * dcolor_base[ch];
          dY[k] += shi[3 * k + ch] * dcolor_base[ch];
        }
      }
      /* per-level colours with their own DC also depend on the direction
       * through the shared view-dependent part */
      if (fov && fov->dc_lv)
        for (int l = 2; l <= L; ++l) {
          const double *dc = &dcol[((int64_t)(l - 1) * nitems + id) * 3];
          for (int ch = 0; ch < 3; ++ch) {
            double raw = it->rest[ch] + Y00 * fov->dc_lv[((int64_t)(l - 2) * n + i) * 3 + ch] + SH_OFFSET;
            if (!(raw > 0.0)) continue;
            for (int k = 1; k < S; ++k) dY[k] += shi[3 * k + ch] * dc[ch];
          }
        }
      double gY[16][3];
      sh_basis_grad(it->dir, gY);
      double ddir[3] = {0, 0, 0};
      for (int k = 1; k < S; ++k)
        for (int a = 0; a < 3; ++a) ddir[a] += dY[k] * gY[k][a];
      /* dir = (mu - cc) / |mu - cc| */
      double dd = ddir[0] * it->dir[0] + ddir[1] * it->dir[1] + ddir[2] * it->dir[2];
      for (int a = 0; a < 3; ++a) d_means[3 * i + a] += (ddir[a] - dd * it->dir[a]) / it->dist;

      /* conic Q = S2^-1 : dS2 = -Q dQ Q (dQ symmetric, off-diagonal split) */
      double Q[4] = {it->conic[0], it->conic[1], it->conic[1], it->conic[2]};
      double dQ[4] = {g2[id].dconic[0], 0.5 * g2[id].dconic[1], 0.5 * g2[id].dconic[1],
                      g2[id].dconic[2]};
      double tmp[4], dS2[4];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          tmp[2 * a + b] = dQ[2 * a] * Q[b] + dQ[2 * a + 1] * Q[2 + b];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          dS2[2 * a + b] = -(Q[2 * a] * tmp[b] + Q[2 * a + 1] * tmp[2 + b]);
      /* S2 = T Sig T^T + 0.3 I : dT = 2 dS2 T Sig, dSig = T^T dS2 T */
      double TS[6];
      for (int a = 0; a < 2; ++a)
        for (int k = 0; k < 3; ++k) {
          double acc = 0.0;
          for (int j = 0; j < 3; ++j) acc += it->T[3 * a + j] * it->Sig[3 * j + k];
          TS[3 * a + k] = acc;
        }
      double dT[6];
      for (int a = 0; a < 2; ++a)
        for (int k = 0; k < 3; ++k)
          dT[3 * a + k] = 2.0 * (dS2[2 * a] * TS[k] + dS2[2 * a + 1] * TS[3 + k]);
      double dSig[9];
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
          double acc = 0.0;
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
              acc += it->T[3 * a + j] * dS2[2 * a + b] * it->T[3 * b + k];
          dSig[3 * j + k] = acc;
        }
      /* Sig = M M^T : dM = (dSig + dSig^T) M */
      double dM[9];
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
          double acc = 0.0;
          for (int l = 0; l < 3; ++l)
            acc += (dSig[3 * j + l] + dSig[3 * l + j]) * it->M[3 * l + k];
          dM[3 * j + k] = acc;
        }
      /* M = Rq diag(s) */
      const double *s3 = &scales[3 * i];
      double dR[9];
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
          d_scales[3 * i + k] += dM[3 * j + k] * it->r[3 * j + k];
          dR[3 * j + k] = dM[3 * j + k] * s3[k];
        }
      /* Rq(q^) with q^ = q / |q| */
      double w = it->qn[0], x = it->qn[1], y = it->qn[2], z = it->qn[3];
      double dqn[4];
      dqn[0] = 2.0 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
      dqn[1] = 2.0 * (y * dR[1] + z * dR[2] + y * dR[3] - 2.0 * x * dR[4] - w * dR[5] +
                      z * dR[6] + w * dR[7] - 2.0 * x * dR[8]);
      dqn[2] = 2.0 * (-2.0 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] -
                      w * dR[6] + z * dR[7] - 2.0 * y * dR[8]);
      dqn[3] = 2.0 * (-2.0 * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.0 * z * dR[4] +
                      y * dR[5] + x * dR[6] + y * dR[7]);
      if (it->qnorm > 0.0) {
        double dot = dqn[0] * w + dqn[1] * x + dqn[2] * y + dqn[3] * z;
        d_quats[4 * i + 0] += (dqn[0] - dot * w) / it->qnorm;
        d_quats[4 * i + 1] += (dqn[1] - dot * x) / it->qnorm;
        d_quats[4 * i + 2] += (dqn[2] - dot * y) / it->qnorm;
        d_quats[4 * i + 3] += (dqn[3] - dot * z) / it->qnorm;
      }
      /* T = J W : dJ = dT W^T */
      double dJ[6];
      for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j) {
          double acc = 0.0;
          for (int k = 0; k < 3; ++k) acc += dT[3 * a + k] * R[3 * j + k];
          dJ[3 * a + j] = acc;
        }
      double px = it->pc[0], py = it->pc[1], pz = it->pc[2];
      double fx = c->fx, fy = c->fy;
      double dpc[3] = {0, 0, 0};
      dpc[2] += dJ[0] * (-fx / (pz * pz)) + dJ[4] * (-fy / (pz * pz)) +
                dJ[2] * (2.0 * fx * it->xcl / (pz * pz * pz)) +
                dJ[5] * (2.0 * fy * it->ycl / (pz * pz * pz));
      double dxcl = dJ[2] * (-fx / (pz * pz));
      double dycl = dJ[5] * (-fy / (pz * pz));
      if (it->clx) dpc[2] += dxcl * it->clx * it->limx; else dpc[0] += dxcl;
      if (it->cly) dpc[2] += dycl * it->cly * it->limy; else dpc[1] += dycl;
      /* mean2D */
      double du = g2[id].dmu2[0], dv = g2[id].dmu2[1];
      dpc[0] += du * fx / pz;
      dpc[1] += dv * fy / pz;
      dpc[2] += -du * fx * px / (pz * pz) - dv * fy * py / (pz * pz);
      for (int a = 0; a < 3; ++a)
        d_means[3 * i + a] += R[a] * dpc[0] + R[3 + a] * dpc[1] + R[6 + a] * dpc[2];
    }
  }
  free(vis); free(vp); free(items); free(g2); free(dop); free(dcol);
  free(g2a); free(dopa); free(dcola);
  return 0;
}
