/*
 * gs_oracle.h -- plain, slow CPU oracle for the tile rasterizer and the
 * foveated multi-level render.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this code; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA path.
 *
 * What it computes (paper: MetaSapiens, arXiv 2407.00435):
 *   * Eq. 1a: p = sum_i T_i alpha_i c_i with T_i = prod_{j<i}(1 - alpha_j),
 *     over the ellipses intersecting the pixel, near to far (Sec. 2.1).
 *   * Eq. 1b/1c: alpha_i = f(opacity, pose), c_i = g(SH); the paper defers f
 *     and g to the 3D Gaussian Splatting paper, so the readings below are
 *     used (EWA splat with a 0.3 px^2 low-pass, 3-sigma square support,
 *     alpha floor 1/255, alpha clamp 0.99, stop before the point that would
 *     take T below 1e-4, real SH up to degree 3 plus 0.5, clamped at 0).
 *   * Sec. 2.1 projection / sorting: per-tile lists sorted by depth.
 *   * Sec. 4.1-4.2 foveated rendering: quality bound m per point, filtering
 *     of tile/point pairs with t > m, per-level accumulation over nested
 *     subsets, linear blend in a band outside each region boundary,
 *     selective multi-versioning of opacity and SH DC.
 *   * Sec. 3.2 cost statistics: tiles touched / used, pixels blended,
 *     pixels dominated (argmax of T_i alpha_i).
 *
 * Precision: everything that produces a value (2D mean, covariance, conic,
 * colour, alpha, transmittance, gradients) is FP64.  Everything that makes a
 * discrete decision that the GPU must reproduce bit for bit (visibility,
 * depth order, tile rectangle, foveation level of a pixel or tile) is taken
 * in FP32 in the fixed operation order documented beside each function
 * ("keyed" path), compiled without floating-point contraction.
 */
#ifndef GS_ORACLE_H
#define GS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Camera: world->camera rotation R (row-major) and translation t (OpenCV:
 * x right, y down, z forward), pinhole intrinsics, image size, clip range. */
typedef struct {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float znear, zfar;
} orc_cam;

/* Foveation description shared by all views of one call. */
typedef struct {
  int32_t n_levels;          /* L >= 1 */
  const uint8_t *bound_m;    /* (N,)  quality bound m in 1..L */
  const float *ring_tan;     /* (L-1,) tan(eccentricity) of region boundaries */
  float band_px;             /* blend band width outside each boundary, px */
  const float *gaze;         /* (V,2) gaze pixel per view */
  const uint8_t *view_fov;   /* (V,) 1 = foveated, 0 = plain; NULL = all foveated */
  const double *opacity_lv;  /* (L-1,N) opacity of levels 2..L, or NULL */
  const double *dc_lv;       /* (L-1,N,3) SH DC of levels 2..L, or NULL */
  int32_t disjoint;          /* 0: nested subsets, level l uses the points with m >= l
                                (Sec. 4.2); 1: a separate model per level (Sec. 4.1),
                                bound_m = the level of the model a point belongs to and
                                level l uses exactly the points with m == l */
} orc_fov;

/* Per-item (view, point) FP64 value record produced by orc_project_values. */
enum {
  ORC_U = 0, ORC_V, ORC_CA, ORC_CB, ORC_CC,   /* mean2D, conic (a b; b c) */
  ORC_R, ORC_G, ORC_B,                         /* colour after clamp */
  ORC_RR, ORC_RG, ORC_RB,                      /* view-dependent part (l >= 1) */
  ORC_DEPTH, ORC_SA, ORC_SB, ORC_SC,           /* camera z, 2D covariance */
  ORC_NVAL                                     /* = 15 */
};

/* Keyed projection (FP32, fixed order).  For each view v and point i writes
 * vis[v*N+i] (1 visible, 0 culled, 2 culled because a parameter is not
 * finite), depth_bits (raw bits of the camera z), rect = {x0, x1, y0, y1}
 * inclusive tile bounds (only meaningful when visible).  supp (nullable,
 * 6 floats per item: keyed 2D mean, 2D covariance a b c, tau) receives
 * the opacity-aware tight support of each visible item; fov (nullable) only
 * supplies the per-level opacities that support must cover.  Returns 0. */
int orc_keyed_project(int n, const float *means, const float *scales,
                      const float *quats, const float *opac, const float *sh,
                      int sh_degree, int V, const orc_cam *cams, int tile,
                      const orc_fov *fov, uint8_t *vis, uint32_t *depth_bits,
                      int32_t *rect, float *supp);

/* Per-tile filter level (FP32 keyed): minimum over the tile's pixels of
 * the lowest level that pixel needs.  Tiles of plain views get 1.
 * Tiles are numbered view by view, row-major inside a view. */
int orc_tile_levels(int V, const orc_cam *cams, int tile, const orc_fov *fov,
                    uint8_t *tile_level);

/* Total tiles of all views. */
int64_t orc_total_tiles(int V, const orc_cam *cams, int tile);

/* Pair count K.  counts[v*N+i] receives the number of kept tile pairs: the
 * tiles of the rectangle that pass the foveation filter and, when supp is
 * given, meet the tight support. */
int64_t orc_count_pairs(int n, int V, const orc_cam *cams, int tile,
                        const uint8_t *vis, const int32_t *rect,
                        const uint8_t *tile_level, const uint8_t *bound_m,
                        const float *supp, uint32_t *counts);

/* Emit the K pairs in (view, point, tile-row, tile-col) order with key
 * (global tile << 32 | depth bits) and value v*N+i, stable-sort them by key
 * and write per-tile [start, end) ranges (2 uint32 per tile). */
int orc_bin(int n, int V, const orc_cam *cams, int tile, const uint8_t *vis,
            const uint32_t *depth_bits, const int32_t *rect,
            const uint8_t *tile_level, const uint8_t *bound_m, const float *supp,
            int64_t K, uint64_t *keys, uint32_t *vals, uint32_t *ranges);

/* FP64 value projection of every visible item into out[(v*N+i)*ORC_NVAL]. */
int orc_project_values(int n, const double *means, const double *scales,
                       const double *quats, const double *sh, int sh_degree,
                       int V, const orc_cam *cams, const uint8_t *vis,
                       double *out);

/* Real spherical harmonics basis (16 values, degree <= 3) at unit dir. */
void orc_sh_basis(const double dir[3], double Y[16]);

/* Composite pixels (Eq. 1) from the binned lists.
 *   pix      : list of global pixel ids to compute (NULL = all, in order);
 *              global id = pixel offset of the view + y*W + x
 *   rgb      : (npix,3)  C + T*bg (blended in the band for foveated views)
 *   T, last  : (npix,2)  final transmittance and tile-list position of the
 *              last blended point for accumulator A (the pixel's own level)
 *              and B (the next better level, only inside a band; else 1,-1)
 *   margin   : (npix,)   smallest relative distance of any alpha-floor,
 *              alpha-clamp or early-stop decision from its threshold (the
 *              clamp leaves the colour continuous but switches gradients)
 *   wband    : (npix,)   blend weight w of accumulator A (1 outside bands)
 *   ambB     : (npix,)   bound on what flipping the pixel's ambiguous
 *              decisions can change in any channel (0 if none); see the
 *              error model beside composite() in gs_oracle.c
 *   amb      : (npix,)   1 if some alpha-floor or stop decision lies inside
 *              the uncertainty window of an FP32 evaluation
 *   stats    : (4,N) uint32 or NULL: tiles_touched, tiles_used,
 *              pixels_blended, pixels_dominated (accumulator A); only
 *              meaningful when pix == NULL (the whole batch).
 * opac is the (N,) base opacity; fov may be NULL (all views plain). */
int orc_render(int n, int V, const orc_cam *cams, int tile,
               const double *vals_proj, const double *opac,
               const uint32_t *vals, const uint32_t *ranges,
               const orc_fov *fov, const double bg[3],
               const int64_t *pix, int64_t npix, double *rgb, double *T,
               int32_t *last, double *margin, double *wband, double *ambB,
               uint8_t *amb, uint32_t *stats);

/* Brute force of Eq. 1 by its per-pixel definition: each pixel scans every
 * point (no tile lists, no foveation tile filter).  Support = visible and the
 * pixel's tile inside the point's rectangle; order = (FP32 depth, point
 * index); the pixel's level decides which points take part.  Same rgb and T
 * as orc_render; last holds the ITEM (v*N + i) of the last blended point of
 * each accumulator (-1 if none) instead of a list position. */
int orc_render_brute(int n, int V, const orc_cam *cams, int tile,
                     const uint8_t *vis, const uint32_t *depth_bits,
                     const int32_t *rect, const double *vals_proj,
                     const double *opac, const orc_fov *fov,
                     const double bg[3], double *rgb, double *T,
                     int32_t *last);

/* Magnitude of the terms behind each gradient element (test bookkeeping):
 * the same chain as the gradient with every product and sum taken in
 * absolute value, i.e. sum |t| over the terms t whose sum is the element.
 * A finite-precision evaluation errs by about its relative rounding times
 * this, however much the terms cancel.  Arrays as the gradients', each
 * nullable. */
typedef struct {
  double *means, *scales, *quats, *opac, *sh, *opac_lv, *dc_lv;
} orc_grad_mag;

/* Analytic FP64 gradient of L = sum(dL_drgb * rgb) with respect to the scene
 * parameters, holding the binning fixed.  Output arrays are overwritten.
 * d_opac_lv / d_dc_lv may be NULL (then fov->opacity_lv must be NULL).
 * mag (nullable) receives the term magnitudes. */
int orc_backward(int n, const double *means, const double *scales,
                 const double *quats, const double *opac, const double *sh,
                 int sh_degree, int V, const orc_cam *cams, int tile,
                 const uint32_t *vals, const uint32_t *ranges,
                 const orc_fov *fov, const double bg[3],
                 const double *dL_drgb, double *d_means, double *d_scales,
                 double *d_quats, double *d_opac, double *d_sh,
                 double *d_opac_lv, double *d_dc_lv, const orc_grad_mag *mag);

#ifdef __cplusplus
}
#endif
#endif
