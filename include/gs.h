/*
 * gs.h -- C ABI of the GB300 (sm_103a) tile rasterizer for point-based
 * neural rendering (3D Gaussian splatting) with foveated multi-level
 * rendering, after MetaSapiens (arXiv 2407.00435).
 *
 * Pipeline (Sec. 2.1 "General PBNR Pipeline", Fig. 1; foveated version
 * Sec. 4.1, Fig. 7E):
 *
 *   gs_project         Projection: each point's ellipsoid is splatted to an
 *                      ellipse on the image plane (2D mean, 2D covariance,
 *                      depth, view-dependent SH colour g, tile rectangle).
 *                      With foveation, the Filtering stage's tile levels
 *                      are computed here too (Sec. 4.2).
 *   gs_bin_sort        Sorting: per tile, the intersecting ellipses ordered
 *                      by depth, near to far (tile/point pairs, radix sort,
 *                      per-tile ranges); foveated pairs with t > m dropped.
 *   gs_render          Rasterization: Eq. 1a per pixel, front to back.
 *   gs_render_fov      Rasterization of foveated views: each pixel composites
 *                      the nested subset of its quality level, pixels in a
 *                      band outside a region boundary also composite the next
 *                      better level and the two colours are blended
 *                      (Sec. 4.1 "Main Pipeline", Sec. 4.2 multi-versioning).
 *   gs_render_backward Adjoint of the above for retraining through the
 *                      renderer (Sec. 3.4, Sec. 4.3).
 *
 * Conventions shared by every entry point:
 *   * Pointers named *_dev or documented as "device" are CUDA device
 *     memory owned by the caller; the library never frees or keeps them
 *     beyond what gs_project records in the plan (the scene and camera
 *     pointers, which must stay valid until the last call that uses them).
 *   * The library allocates nothing.  All scratch lives in the caller's
 *     workspace (size from gs_workspace_size) and in the caller's host-side
 *     plan buffer (size from gs_plan_size).
 *   * Every call is asynchronous on the given stream and returns as soon as
 *     its kernels are enqueued; host-side argument errors return at once
 *     and enqueue nothing.  No call synchronises except gs_get_error.
 *   * Device-side problems (pair capacity exceeded, a bounded wait that gave
 *     up) are recorded in a sticky status word inside the workspace and
 *     reported by gs_get_error.  No exception crosses the ABI.
 *   * Points with a non-finite parameter are culled and counted.
 *   * Outputs are overwritten, never accumulated; gradient outputs are
 *     zeroed by gs_render_backward itself.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gs_status;
#define GS_OK 0
#define GS_ERR_INVALID_ARG 1 /* bad host-side argument; nothing enqueued */
#define GS_ERR_CAPACITY 2    /* more tile/point pairs than the plan holds */
#define GS_ERR_TIMEOUT 3     /* a bounded device-side wait gave up */
#define GS_ERR_CUDA 4        /* a CUDA runtime call failed */
#define GS_ERR_UNSUPPORTED 5 /* valid but not supported (e.g. SH degree > 3) */

/* Pinhole camera, world -> camera: p_c = R p_w + t, OpenCV axes (x right,
 * y down, z forward).  Pixel (x, y) has its centre at (x + 0.5, y + 0.5);
 * the projected mean of p_c is (fx x/z + cx, fy y/z + cy).  Points with
 * z <= znear or z >= zfar are culled.  80 bytes, no padding. */
typedef struct gs_camera {
  float R[9]; /* row-major */
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float znear, zfar;
} gs_camera;

/* The scene: the trainable parameters of each point listed in Sec. 2.1
 * (position, scales, orientation, opacity, SH colour).  All device, fp32,
 * C-contiguous. */
typedef struct gs_scene {
  int64_t n;          /* number of points N */
  int32_t sh_degree;  /* 0..3; S = (sh_degree + 1)^2 coefficients */
  int32_t reserved;
  const float *means;     /* (N,3) world positions */
  const float *scales;    /* (N,3) per-axis std, already activated (> 0) */
  const float *quats;     /* (N,4) rotation (w,x,y,z), any length; 0 -> identity */
  const float *opacities; /* (N,)  already activated, in (0,1) */
  const float *sh;        /* (N,S,3) SH coefficients, RGB innermost */
} gs_scene;

#define GS_MAX_LEVELS 8

/* Foveation (Sec. 4.1-4.2).  Quality level 1 is the best.  A pixel at
 * distance d (pixels) from the gaze point has level 1 + #{k : d >= R_k}
 * with ring radius R_k = fy * ring_tan[k] (eccentricity boundary k of L-1,
 * ascending).  Pixels with R_k <= d < R_k + band_px (boundary k, level
 * k+1) also composite level k and output
 *   w C_{k+1} + (1 - w) C_k,  w = (d - R_k) / band_px.
 * Level l composites the points whose quality bound m >= l (nested
 * subsets).  A tile's filter level is the smallest level any of its pixels
 * needs; a pair (tile, point) is kept iff tile level <= m. */
typedef struct gs_fov {
  int32_t n_levels;            /* L, 1..GS_MAX_LEVELS */
  float band_px;               /* >= 0 */
  float ring_tan[GS_MAX_LEVELS - 1]; /* host values, L-1 used, ascending */
  const uint8_t *bound_m;      /* device (N,) quality bound m in 1..L */
  const float *gaze_px;        /* device (V,2) gaze pixel per view */
  const uint8_t *view_fov;     /* device (V,) 1 foveated / 0 plain; NULL = all foveated */
  const float *opacity_lv;     /* device (L-1,N) opacity of levels 2..L, or NULL */
  const float *dc_lv;          /* device (L-1,N,3) SH DC of levels 2..L, or NULL */
} gs_fov;
/* Per-level parameters (selective multi-versioning, Sec. 4.2) are supported
 * for L <= 4; gs_project returns GS_ERR_UNSUPPORTED beyond. */

/* Plan options.  Zero-initialised fields take the defaults given. */
typedef struct gs_config {
  int32_t tile;          /* tile edge in pixels: 16 (default) or 8 */
  int32_t chunk;         /* heavy-tile chunk length in points, 64..2^24; <= 0 = whole
                            tiles (default).  See gs_render. */
  int32_t flags;         /* GS_FLAG_* */
  int32_t max_levels;    /* largest foveation L the plan must hold; 0 = 4 */
  int32_t radix_bits;    /* digit width of the pair sort's passes, 4..10 (9 and 10 need the
                            cooperative sort, else 8 is used); 0 = balanced <= 8 */
  int32_t chunk_slots;   /* chunk slots the workspace holds for the chunked render;
                            0 = enough for any split (capped at max(tiles + 64, 65536)).
                            Tiles that do not fit are rendered whole. */
  int64_t max_pairs;     /* capacity of tile/point pairs; 0 = 4 * N * V */
  int32_t wait_spins;    /* polls of gs_project's bounded bulk-copy waits before they give
                            up with GS_ERR_TIMEOUT: 0 = default (2^20 polls, about a
                            second); < 0 = give up without polling (exercises the failure
                            path; the frame's records are then incomplete, see gs_project) */
  int32_t reserved;
} gs_config;

#define GS_FLAG_FOVEATED 1u  /* reserve foveation state (levels, per-level params) */
#define GS_FLAG_BACKWARD 2u  /* reserve per-item gradient scratch for gs_render_backward */
#define GS_FLAG_TIGHT 4u     /* opacity-aware tight support: of each point's 3-sigma tile
                                rectangle keep only the tiles whose pixel-centre rectangle
                                meets the ellipse where alpha can reach 1/255 (an upper
                                bound of 2 ln(255 o) on the Mahalanobis distance, o the
                                largest opacity of any level).  Same image, shorter tile
                                lists.  Rectangles of more than 256 tiles keep all tiles. */
#define GS_FLAG_MULTI_MODEL 8u  /* foveated render with a separate model per quality level
                                (Sec. 4.1, main pipeline): the scene is the concatenation of
                                the levels' models and gs_fov.bound_m holds the level of the
                                model each point belongs to.  A pixel of level l composites
                                only the points of model l (and, inside a blend band, those
                                of model l - 1 into its second accumulator).  Requires
                                GS_FLAG_FOVEATED, a gs_fov in every gs_project and
                                gs_render_fov; per-level parameters (opacity_lv, dc_lv) are
                                rejected (every model carries its own). */

/* Counters read back by gs_get_error. */
typedef struct gs_counters {
  uint32_t status;       /* sticky device status (GS_OK, GS_ERR_CAPACITY, GS_ERR_TIMEOUT) */
  uint32_t reserved;
  uint64_t n_visible;    /* visible (view, point) items M */
  uint64_t n_pairs;      /* tile/point pairs K (before any capacity clamp) */
  uint64_t n_nonfinite;  /* (view, point) items culled for a non-finite parameter */
  uint64_t n_evals;      /* (pixel, point) alpha evaluations of the last render with stats */
  uint64_t n_blends;     /* of which blended (alpha >= 1/255, before the stop) */
} gs_counters;

/* Opaque host-side plan, caller-allocated with gs_plan_size() bytes
 * (8-byte aligned).  Holds sizes, workspace offsets and the pointers given
 * to gs_project; contains no device memory of its own. */
typedef struct gs_plan gs_plan;

size_t gs_plan_size(void);

/* Fill a plan for N points of SH degree sh_degree rendered into n_views
 * views.  cams_host (host memory, n_views entries) fixes the image sizes;
 * later calls must pass device cameras of the same sizes (poses may
 * change).  cfg may be NULL.  Errors: GS_ERR_INVALID_ARG (sizes, tile),
 * GS_ERR_UNSUPPORTED (sh_degree > 3). */
gs_status gs_plan_init(gs_plan *plan, int64_t n, int32_t sh_degree,
                       const gs_camera *cams_host, int32_t n_views,
                       const gs_config *cfg);

/* Bytes of device workspace the plan needs (256-byte aligned base). */
size_t gs_workspace_size(const gs_plan *plan);

/* Projection (+ FR tile levels).  scene: device arrays; cams_dev: device
 * array of n_views gs_camera; fov: NULL for plain rendering, else the
 * foveation of every view (requires GS_FLAG_FOVEATED).  Records the scene,
 * camera and fov in the plan for the calls below.  The point parameters are
 * staged by bulk copies whose waits are bounded (gs_config.wait_spins); a
 * wait that gives up sets GS_ERR_TIMEOUT and leaves that block's records
 * unwritten, so a caller that sees GS_ERR_TIMEOUT from gs_get_error after
 * gs_project must project again before gs_bin_sort.
 * Errors: GS_ERR_INVALID_ARG (NULL pointer, ws too small or unaligned,
 * n mismatch, bad fov), GS_ERR_CUDA. */
gs_status gs_project(gs_plan *plan, void *ws, size_t ws_bytes,
                     const gs_scene *scene, const gs_camera *cams_dev,
                     const gs_fov *fov, cudaStream_t stream);

/* Sorting: emit (tile, point) pairs of the visible items in depth order,
 * stable radix sort by tile, per-tile ranges and the render work list.
 * ws: the workspace gs_project was given (256-byte aligned, else
 * GS_ERR_INVALID_ARG).  Device-side capacity overflow sets GS_ERR_CAPACITY
 * (pairs beyond the capacity are dropped, nothing is written out of
 * bounds). */
gs_status gs_bin_sort(gs_plan *plan, void *ws, cudaStream_t stream);

/* Rasterization of plain views (Eq. 1a) with the readings: alpha =
 * min(0.99, o exp(-1/2 d^T Sigma'^-1 d)), points with alpha < 1/255
 * skipped, compositing stops before the point that would take T below
 * 1e-4.  Outputs (device, pixels of all views concatenated view by view,
 * row-major inside a view):
 *   rgb     (P,3)  C + T bg
 *   T_final (P,)   final transmittance
 *   last    (P,)   position, inside the pixel's tile list, of the last
 *                  blended point (-1 if none)
 *   stats   (4,N)  uint32 or NULL: tiles_touched, tiles_used,
 *                  pixels_blended, pixels_dominated, summed over the views
 *                  (cost statistics of Sec. 3.2: Comp_i and Val_i).
 * bg is host memory (3 floats).  All views of the plan must be plain (the
 * plan's fov, if any, is ignored).
 * Work distribution: with the plan's chunk <= 0 one block composites each
 * tile.  With chunk > 0 persistent blocks take work from a queue: a tile
 * with more than `chunk` pairs is split into chunks composited in parallel
 * from T = 1 and merged in list order by (C1, T1) o (C2, T2) = (C1 + T1 C2,
 * T1 T2); the chunk in which the early stop falls is re-walked from the
 * incoming transmittance, so the stop rule above holds exactly.  Renders
 * with stats always walk whole tiles.  Results agree to float rounding. */
gs_status gs_render(gs_plan *plan, void *ws, const float bg[3], float *rgb,
                    float *T_final, int32_t *last, uint32_t *stats,
                    cudaStream_t stream);

/* Rasterization with the fov given to gs_project (views with view_fov = 0
 * render plain).  T_final and last have two entries per pixel: [0] for the
 * pixel's own level, [1] for the better level inside a blend band (1 and
 * -1 elsewhere).  stats count the pixel's own level. */
gs_status gs_render_fov(gs_plan *plan, void *ws, const float bg[3], float *rgb,
                        float *T_final, int32_t *last, uint32_t *stats,
                        cudaStream_t stream);

/* Adjoint of the last gs_render / gs_render_fov of this plan for the loss
 * sum(dL_drgb * rgb).  T_final and last are that call's outputs (same
 * layout); bg the same background.  Gradients (device, fp32, overwritten):
 * d_means (N,3), d_scales (N,3), d_quats (N,4), d_opac (N,), d_sh (N,S,3),
 * d_opac_lv (L-1,N) and d_dc_lv (L-1,N,3) (may be NULL when the fov has no
 * per-level parameters).  Requires GS_FLAG_BACKWARD. */
gs_status gs_render_backward(gs_plan *plan, void *ws, const float *dL_drgb,
                             const float *T_final, const int32_t *last,
                             const float bg[3], float *d_means, float *d_scales,
                             float *d_quats, float *d_opac, float *d_sh,
                             float *d_opac_lv, float *d_dc_lv,
                             cudaStream_t stream);

/* Synchronise `stream`, read the device status word and counters.  Returns
 * the device status (GS_OK if nothing went wrong); out may be NULL.  The
 * status word is reset by gs_project and then keeps the first device-side
 * error of the frame (project, bin_sort, render, backward). */
gs_status gs_get_error(const gs_plan *plan, const void *ws, cudaStream_t stream,
                       gs_counters *out);

/* Clear the sticky device status word (asynchronous). */
gs_status gs_clear_error(const gs_plan *plan, void *ws, cudaStream_t stream);

/* Location of a workspace region, for tests and debugging.  region is one
 * of GS_REGION_*; offset and bytes are relative to the workspace base.
 * Every (view v, point i) owns the item slot j = i * V + v.  Slots of items
 * that are not visible hold depth key 0xffffffff and a zero pair count; the
 * other fields of such slots are unspecified. */
#define GS_REGION_ITEM_GID 1     /* uint32 (N*V) point index of slot j */
#define GS_REGION_ITEM_VIEW 2    /* uint32 (N*V) view of slot j */
#define GS_REGION_ITEM_DEPTH 3   /* uint32 (N*V) float bits of camera z */
#define GS_REGION_ITEM_COUNT 4   /* uint32 (N*V) kept tile pairs of slot j */
#define GS_REGION_RANGES 7       /* uint32 (T,2) [start, end) per global tile */
#define GS_REGION_TILE_LEVEL 8   /* uint8  (T)  FR filter level per global tile */
gs_status gs_ws_region(const gs_plan *plan, int32_t region, size_t *offset,
                       size_t *bytes);

/* Device pointers to the K sorted pairs of the last gs_bin_sort: global
 * tile id and visible item j of each pair, ordered by (tile, depth, point
 * index).  Synchronises `stream` (the sort picks its output buffer on the
 * device).  Pointers stay valid until the next gs_bin_sort.  The item of
 * a pair is its slot j = i * V + v (see GS_REGION_ITEM_*). */
gs_status gs_sorted_pairs(const gs_plan *plan, const void *ws, cudaStream_t stream,
                          const uint32_t **pair_tile, const uint32_t **pair_item);

/* Allocation-free stable radix sort of (key, value) pairs by key, keys
 * below 2^key_bits (key_bits 1..32): the pair sort of gs_bin_sort for
 * callers that cannot allocate device memory -- code inside a memory pool
 * that must not grow, plug-ins whose host application forbids cudaMalloc
 * after start-up, real-time paths where an allocation could block -- and so
 * cannot size a workspace.  The paper has no counterpart; this is a
 * property of the library only.
 *   keys_in, vals_in   device, n entries each, not modified
 *   keys_out, vals_out device, n entries each, overwritten with the pairs in
 *                      key order (equal keys keep their input order)
 * Scratch is one static device array of this library, sized for at most
 * GS_STATIC_SORT_MAX_PAIRS pairs: 12,587,264 bytes (about 12.6 MB), held on
 * every GPU that loads the library until the process exits.  No call
 * allocates or frees.  The first call on a device looks up the array's
 * device address (a one-time set-up); make that first call before any
 * stream capture.  All calls of this process on one device share the array
 * and it keeps the last call's contents: calls that may overlap on the GPU
 * (for example on different streams) race and must be serialised by the
 * caller.  A device-side failure (a bounded wait that gave up, leaving the
 * output incomplete) is recorded in the array's status word: read it with
 * gs_sort_pairs_static_status after the call.  Errors: GS_ERR_INVALID_ARG
 * (n < 0 or n > GS_STATIC_SORT_MAX_PAIRS, key_bits out of range, NULL or
 * overlapping buffers), GS_ERR_CUDA. */
#define GS_STATIC_SORT_MAX_PAIRS (1 << 20)
gs_status gs_sort_pairs_static(const uint32_t *keys_in, const uint32_t *vals_in,
                               int64_t n, int32_t key_bits, uint32_t *keys_out,
                               uint32_t *vals_out, cudaStream_t stream);

/* Device status of the last gs_sort_pairs_static on the current device:
 * synchronises `stream` (the stream of that call), writes the status word
 * (GS_OK, or GS_ERR_TIMEOUT when a bounded wait gave up and the output is
 * incomplete) to *host_status (host memory) and returns it.  GS_OK when no
 * such sort ran on this device.  Allocates nothing.  Errors:
 * GS_ERR_INVALID_ARG (NULL host_status), GS_ERR_CUDA. */
gs_status gs_sort_pairs_static_status(uint32_t *host_status, cudaStream_t stream);

/* 1 if, on the current device, each radix sort of gs_bin_sort (and of
 * gs_prune_mask, gs_sort_pairs_static) runs as one cooperative launch of one
 * block per SM whose passes are separated by bounded grid barriers; 0 if it
 * runs as three launches per pass (cooperative launch unavailable).  For
 * launch accounting; no counterpart in the paper. */
int32_t gs_sort_is_cooperative(void);

/* Geometry helpers (host): total tiles and pixels of the plan's views. */
int64_t gs_plan_tiles(const gs_plan *plan);
int64_t gs_plan_pixels(const gs_plan *plan);

/* ---- efficiency-aware pruning and scale decay (Sec. 3.2-3.4) ---------- */

/* Computational efficiency of each point in one pose (Sec. 3.2, Eq. 2):
 * CE_i = Val_i / Comp_i with Val_i = pixels dominated by the point and
 * Comp_i = tiles whose list holds it (tiles_touched), both from the stats
 * buffer (4,N) of a gs_render / gs_render_fov call on that pose.  Keeps the
 * maximum over poses: ce_max[i] = max(ce_max[i], CE_i); points no tile
 * holds leave ce_max[i] unchanged.  ce_max: device (N,) float, zeroed by the
 * caller before the first pose.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
gs_status gs_ce_update(int64_t n, const uint32_t *stats, float *ce_max, cudaStream_t stream);

/* Intersection-aware pruning (Sec. 3.2; R = 10% per round in Sec. 3.4):
 * keep[i] = 0 for the floor(fraction * n) points with the lowest ce_max
 * (ties: lower index first), 1 for the others.  ce_max (device, n
 * non-negative floats) is sorted with its indices in the plan's depth-sort
 * buffers, so n must not exceed the plan's item slots (N x V); the last
 * gs_bin_sort's depth order is overwritten (rendering needs a new
 * gs_project / gs_bin_sort).  fraction in [0, 1].  keep: device (n,) bytes. */
gs_status gs_prune_mask(gs_plan *plan, void *ws, int64_t n, const float *ce_max, double fraction,
                        uint8_t *keep, cudaStream_t stream);

/* Stable compaction of a scene by keep (device (n,) bytes): the kept points'
 * parameters are copied, in order, from `in` to `out` (device arrays with
 * room for n points, not overlapping `in`); *n_out (device uint64) receives
 * the number kept.  Uses the plan's workspace as scratch (any plan). */
gs_status gs_compact_points(gs_plan *plan, void *ws, int64_t n, int32_t sh_degree,
                            const uint8_t *keep, const gs_scene *in, gs_scene *out,
                            uint64_t *n_out, cudaStream_t stream);

/* Weighted scale (Sec. 3.3, Eq. 3-4): WS = (1/N) sum_i S_i G_i with S_i the
 * largest of point i's three (activated) scales and G_i = (U_i > T)(U_i - T),
 * U_i = tiles where the point was blended (tiles_used, stats row 1).  Writes
 * WS to *ws_out (device double) and, if d_scales is given, adds
 * gamma dWS/ds (gamma G_i / N on the first largest axis) to it, the scale
 * decay term of the loss L = L_quality + gamma WS (Eq. 5). */
gs_status gs_weighted_scale(int64_t n, const float *scales, const uint32_t *stats, float T,
                            float gamma, double *ws_out, float *d_scales, cudaStream_t stream);

/* ---- eccentricity-aware quality (HVSQ) ---------------------------------- */

/* Bytes of device scratch gs_hvsq needs for a width x height image
 * (18 FP64 planes of (width + 1) x (height + 1) plus accumulators); 0 for
 * bad sizes. */
size_t gs_hvsq_scratch_size(int32_t width, int32_t height);

/* HVSQ of an altered image against a reference (Sec. 2.2, the HVSQ
 * equation), per quality region (Sec. 4.3), and optionally its gradient:
 *   HVSQ_g = (1/N_g) sum over the N_g pixels i of region g of
 *            sum_c (mean_c(a, P_i) - mean_c(r, P_i))^2
 *                  + (std_c(a, P_i) - std_c(r, P_i))^2
 * with P_i the square box of half-width r_i around pixel i clipped to the
 * image, mean / std (population) over the box per colour channel c.
 * Geometry (FP32, the renderer's ring test): d_i^2 = (x + 0.5 - gaze_x)^2 +
 * (y + 0.5 - gaze_y)^2; r_i = r_base + #{j : d_i^2 >= (focal pool_tan[j])^2}
 * (the pooling grows with eccentricity: pool_tan are the tangents of the
 * eccentricities where it gains a pixel, ascending, n_pool <= 64); region
 * g_i = #{k : d_i^2 >= (focal ring_tan[k])^2} (quality level - 1; n_rings
 * <= 7, 0 = one region).
 *   alt, ref  device (width*height, 3) fp32, row-major (a gs_render image)
 *   ring_tan, pool_tan  host arrays
 *   scratch   device, gs_hvsq_scratch_size bytes, 256-byte aligned
 *   hvsq_out  device, n_rings + 1 doubles, written
 *   d_alt     device (width*height, 3) fp32 or NULL: gradient of the sum of
 *             the regions' HVSQs with respect to alt (overwritten); at a
 *             pooling whose std is 0 the std term contributes 0 (subgradient)
 * Asynchronous on `stream`.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
gs_status gs_hvsq(const float *alt, const float *ref, int32_t width, int32_t height,
                  float gaze_x, float gaze_y, float focal, const float *ring_tan,
                  int32_t n_rings, const float *pool_tan, int32_t n_pool, int32_t r_base,
                  void *scratch, size_t scratch_bytes, double *hvsq_out, float *d_alt,
                  cudaStream_t stream);

/* ---- measurement -------------------------------------------------------- */

/* Issue-rate probe of the two units the render is bound by (the roofline
 * denominators; no counterpart in the paper): kind 0 runs chains of
 * independent FP32 fused multiply-adds, kind 1 chains of ex2.approx on the
 * special-function unit, on every resident thread of every SM, `iters`
 * steps of 8 chains per thread.  *ops (host) receives the lane operations
 * launched (one FMA or one ex2 = one), so the caller divides it by the
 * call's event-timed duration.  d_sink: device float receiving a checksum
 * (keeps the work alive).  Errors: GS_ERR_INVALID_ARG (kind, iters < 1,
 * NULL pointers), GS_ERR_CUDA. */
gs_status gs_peak_probe(int32_t kind, int32_t iters, float *d_sink, int64_t *ops,
                        cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
