// gs_api.cu -- host side of the C ABI declared in include/gs.h: plan and
// workspace layout, argument validation, and the launch sequence of each
// stage.  Nothing here allocates device or host memory.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "gs_internal.cuh"

using namespace gs;

namespace {

constexpr uint64_t kPlanMagic = 0x67735f706c616e31ull;  // "gs_plan1"

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool plan_ok(const gs_plan *p) { return p && p->magic == kPlanMagic; }

gs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

int ceil_log2(long long x) {
  int b = 0;
  while ((1ll << b) < x) ++b;
  return b < 1 ? 1 : b;
}

}  // namespace

extern "C" {

size_t gs_plan_size(void) { return sizeof(gs_plan); }

gs_status gs_plan_init(gs_plan *p, int64_t n, int32_t sh_degree, const gs_camera *cams,
                       int32_t V, const gs_config *cfg) {
  if (!p || !cams || V < 1 || V > kMaxViews || n < 0 || n > 0xffffffffll) return GS_ERR_INVALID_ARG;
  if (sh_degree < 0) return GS_ERR_INVALID_ARG;
  if (sh_degree > 3) return GS_ERR_UNSUPPORTED;
  gs_config c = {};
  if (cfg) c = *cfg;
  if (c.tile == 0) c.tile = 16;
  if (c.tile != 16 && c.tile != 8) return GS_ERR_INVALID_ARG;
  int max_levels = c.max_levels > 0 ? c.max_levels : 4;
  if (max_levels > GS_MAX_LEVELS) return GS_ERR_INVALID_ARG;
  memset(p, 0, sizeof(*p));
  p->n = n;
  p->sh_degree = sh_degree;
  p->V = V;
  p->tile = c.tile;
  if (c.chunk > 0 && (c.chunk < 64 || c.chunk > (1 << 24))) return GS_ERR_INVALID_ARG;
  p->chunk = c.chunk > 0 ? c.chunk : 0;
  if (c.radix_bits != 0 && (c.radix_bits < 4 || c.radix_bits > 10)) return GS_ERR_INVALID_ARG;
  p->radix_bits = c.radix_bits;
  if (((uint32_t)c.flags & GS_FLAG_MULTI_MODEL) && !((uint32_t)c.flags & GS_FLAG_FOVEATED))
    return GS_ERR_INVALID_ARG;
  if ((uint32_t)c.flags &
      ~(GS_FLAG_FOVEATED | GS_FLAG_BACKWARD | GS_FLAG_TIGHT | GS_FLAG_MULTI_MODEL))
    return GS_ERR_INVALID_ARG;
  p->flags = (uint32_t)c.flags;
  p->wait_spins = c.wait_spins;
  long long tiles = 0, pixels = 0, rows = 0;
  for (int v = 0; v < V; ++v) {
    const gs_camera &cam = cams[v];
    if (cam.width <= 0 || cam.height <= 0) return GS_ERR_INVALID_ARG;
    long long tx = (cam.width + c.tile - 1) / c.tile, ty = (cam.height + c.tile - 1) / c.tile;
    if (tx > 65535 || ty > 65535) return GS_ERR_INVALID_ARG;
    tiles += tx * ty;
    rows += ty;
    pixels += (long long)cam.width * cam.height;
    if (cam.width > p->max_w) p->max_w = cam.width;
    if (cam.height > p->max_h) p->max_h = cam.height;
  }
  if (tiles > 0xffffffffll) return GS_ERR_INVALID_ARG;
  p->tiles_total = tiles;
  p->rows_total = rows;
  p->pixels_total = pixels;
  long long items = n * (long long)V;
  // records live at fixed slots i * V + v, so every (view, point) has one
  p->max_visible = items;
  if (p->max_visible > 0xffffffffll) return GS_ERR_INVALID_ARG;   // slots are uint32
  long long mp = c.max_pairs > 0 ? c.max_pairs : 4 * p->max_visible;
  if (mp > 0xfffffffell) mp = 0xfffffffell;
  if (mp < 1) mp = 1;
  p->max_pairs = mp;
  p->tile_bits = ceil_log2(tiles);
  int dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    p->num_sms = 0;
  cudaGetLastError();  // no device (CPU-only host): sizes still valid

  const bool fov = (p->flags & GS_FLAG_FOVEATED) != 0;
  const bool bwd = (p->flags & GS_FLAG_BACKWARD) != 0;
  const long long M = p->max_visible > 0 ? p->max_visible : 1;
  const long long K = p->max_pairs;
  const long long T = tiles > 0 ? tiles : 1;
  size_t b[R_COUNT_] = {};
  b[R_HDR] = sizeof(Hdr);
  b[R_VIEWS] = sizeof(ViewDev) * (size_t)V;
  b[R_TILE_LEVEL] = fov ? (size_t)T : 0;
  b[R_LEVEL_ROWS] = fov ? 4 * (size_t)GS_MAX_LEVELS * (size_t)(rows > 0 ? rows : 1) : 0;
  b[R_REC_MEAN] = b[R_REC_SHAPE] = b[R_REC_COLOR] = 16 * (size_t)M;
  b[R_REC_REST] = fov ? 16 * (size_t)M : 0;
  b[R_REC_DEPTH] = b[R_REC_COUNT] = b[R_REC_GID] = b[R_REC_VIEW] = 4 * (size_t)M;
  b[R_REC_RECT] = 8 * (size_t)M;
  b[R_REC_M] = fov ? (size_t)M : 0;
  const bool tight = (p->flags & GS_FLAG_TIGHT) != 0;
  b[R_REC_SUPP] = tight ? 16 * (size_t)M : 0;
  b[R_REC_SUPP2] = tight ? 8 * (size_t)M : 0;
  b[R_REC_EMIT] = 32 * (size_t)M;
  b[R_REC_CBIG] = 4 * (size_t)M;
  b[R_DKEY_A] = b[R_DKEY_B] = b[R_DVAL_A] = b[R_DVAL_B] = 4 * (size_t)M;
  b[R_OFFSETS] = 4 * (size_t)M;
  b[R_PKEY_A] = b[R_PKEY_B] = b[R_PVAL_A] = b[R_PVAL_B] = 4 * (size_t)K;
  b[R_BIGQ] = 4 * (size_t)M;
  b[R_RANGES] = 8 * (size_t)T;
  // chunked render: a tile of len > chunk pairs takes ceil(len / chunk) <=
  // 2 len / chunk slots, so 2 K / chunk slots always suffice; capped
  // (tiles beyond the cap are rendered whole)
  if (c.chunk_slots < 0) return GS_ERR_INVALID_ARG;
  if (p->chunk > 0) {
    long long cap = 2 * K / p->chunk + 1;
    const long long lim = T + 64 > 65536 ? T + 64 : 65536;
    if (cap > lim) cap = lim;
    if (c.chunk_slots > 0) cap = c.chunk_slots;
    p->chunk_cap = cap;
  }
  const size_t nacc = fov ? 2 : 1;
  const size_t tpx = (size_t)c.tile * (size_t)c.tile;
  b[R_WORK] = 8 * (size_t)p->chunk_cap;
  b[R_CHUNK_TILE] = p->chunk > 0 ? 16 * (size_t)T : 0;
  b[R_CHUNK_PART] = 16 * nacc * tpx * (size_t)p->chunk_cap;
  b[R_CHUNK_LAST] = 4 * nacc * tpx * (size_t)p->chunk_cap;
  // block table of the reduce-then-scan sort (grid <= SMs x resident blocks)
  p->sort_blocks = (p->num_sms > 0 ? p->num_sms : 160) * kSortBlocksPerSm;
  if (p->sort_blocks > kSortMaxBlocks) p->sort_blocks = kSortMaxBlocks;
  b[R_BSUM] = (256 * sizeof(uint32_t) * kSortSub + sizeof(unsigned long long)) * (size_t)p->sort_blocks;
  b[R_GRAD_ITEM] = bwd ? 16 * sizeof(float) * (size_t)M : 0;
  b[R_GRAD_LV] = (bwd && fov) ? 4 * sizeof(float) * (size_t)(max_levels - 1) * (size_t)M : 0;
  size_t off = 0;
  for (int r = 0; r < R_COUNT_; ++r) {
    p->off[r] = off;
    p->bytes[r] = b[r];
    off += align256(b[r]);
  }
  p->ws_bytes = off;
  p->magic = kPlanMagic;
  return GS_OK;
}

size_t gs_workspace_size(const gs_plan *p) { return plan_ok(p) ? p->ws_bytes : 0; }

int64_t gs_plan_tiles(const gs_plan *p) { return plan_ok(p) ? p->tiles_total : -1; }
int64_t gs_plan_pixels(const gs_plan *p) { return plan_ok(p) ? p->pixels_total : -1; }

gs_status gs_ws_region(const gs_plan *p, int32_t region_id, size_t *offset, size_t *bytes) {
  if (!plan_ok(p) || !offset || !bytes) return GS_ERR_INVALID_ARG;
  int r;
  switch (region_id) {
    case GS_REGION_ITEM_GID: r = R_REC_GID; break;
    case GS_REGION_ITEM_VIEW: r = R_REC_VIEW; break;
    case GS_REGION_ITEM_DEPTH: r = R_REC_DEPTH; break;
    case GS_REGION_ITEM_COUNT: r = R_REC_COUNT; break;
    case GS_REGION_RANGES: r = R_RANGES; break;
    case GS_REGION_TILE_LEVEL: r = R_TILE_LEVEL; break;
    default: return GS_ERR_INVALID_ARG;
  }
  *offset = p->off[r];
  *bytes = p->bytes[r];
  return GS_OK;
}

gs_status gs_project(gs_plan *p, void *ws, size_t ws_bytes, const gs_scene *scene,
                     const gs_camera *cams_dev, const gs_fov *fov, cudaStream_t stream) {
  if (!plan_ok(p) || !ws || !scene || !cams_dev) return GS_ERR_INVALID_ARG;
  if (((uintptr_t)ws & 255) != 0 || ws_bytes < p->ws_bytes) return GS_ERR_INVALID_ARG;
  if (scene->n != p->n || scene->sh_degree != p->sh_degree) return GS_ERR_INVALID_ARG;
  if (p->n > 0 && (!scene->means || !scene->scales || !scene->quats || !scene->opacities ||
                   !scene->sh))
    return GS_ERR_INVALID_ARG;
  if (fov) {
    if (!(p->flags & GS_FLAG_FOVEATED)) return GS_ERR_INVALID_ARG;
    const int L = fov->n_levels;
    if (L < 1 || L > GS_MAX_LEVELS || !(fov->band_px >= 0.0f)) return GS_ERR_INVALID_ARG;
    if (!fov->gaze_px || (p->n > 0 && !fov->bound_m)) return GS_ERR_INVALID_ARG;
    for (int k = 0; k < L - 1; ++k) {
      if (!(fov->ring_tan[k] > 0.0f)) return GS_ERR_INVALID_ARG;
      if (k > 0 && !(fov->ring_tan[k] > fov->ring_tan[k - 1])) return GS_ERR_INVALID_ARG;
    }
    if ((p->flags & GS_FLAG_BACKWARD) && (fov->opacity_lv || fov->dc_lv) &&
        p->bytes[R_GRAD_LV] < 4 * sizeof(float) * (size_t)(L - 1) * (size_t)p->max_visible)
      return GS_ERR_INVALID_ARG;
    if ((fov->opacity_lv || fov->dc_lv) && L > kMvMaxLevels) return GS_ERR_UNSUPPORTED;
    if ((p->flags & GS_FLAG_MULTI_MODEL) && (fov->opacity_lv || fov->dc_lv))
      return GS_ERR_INVALID_ARG;
    p->fov = *fov;
    p->has_fov = 1;
    p->fov_mv = (fov->opacity_lv || fov->dc_lv) && L > 1;
  } else {
    if (p->flags & GS_FLAG_MULTI_MODEL) return GS_ERR_INVALID_ARG;   // levels select the models
    memset(&p->fov, 0, sizeof(p->fov));
    p->has_fov = 0;
    p->fov_mv = 0;
  }
  p->scene = *scene;
  p->cams = cams_dev;
  Hdr *hdr = region<Hdr>(p, ws, R_HDR);
  // a new frame: status word, counters and tickets restart
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(Hdr), stream);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  if ((e = launch_views(p, ws, stream)) != cudaSuccess) return GS_ERR_CUDA;
  if ((e = launch_tile_levels(p, ws, stream)) != cudaSuccess) return GS_ERR_CUDA;
  if ((e = launch_project(p, ws, stream)) != cudaSuccess) return GS_ERR_CUDA;
  return GS_OK;
}

gs_status gs_bin_sort(gs_plan *p, void *ws, cudaStream_t stream) {
  if (!plan_ok(p) || !ws || !p->cams) return GS_ERR_INVALID_ARG;
  if (((uintptr_t)ws & 255) != 0) return GS_ERR_INVALID_ARG;   // (16-byte vector and bulk accesses)
  return cuda_status(launch_bin_sort(p, ws, stream));
}

gs_status gs_render(gs_plan *p, void *ws, const float bg[3], float *rgb, float *T_final,
                    int32_t *last, uint32_t *stats, cudaStream_t stream) {
  if (!plan_ok(p) || !ws || !bg || !rgb || !T_final || !last || !p->cams) return GS_ERR_INVALID_ARG;
  if (p->flags & GS_FLAG_MULTI_MODEL) return GS_ERR_INVALID_ARG;   // gs_render_fov selects the models
  p->last_fov = 0;
  return cuda_status(launch_render(p, ws, false, bg, rgb, T_final, last, stats, stream));
}

gs_status gs_render_fov(gs_plan *p, void *ws, const float bg[3], float *rgb, float *T_final,
                        int32_t *last, uint32_t *stats, cudaStream_t stream) {
  if (!plan_ok(p) || !ws || !bg || !rgb || !T_final || !last || !p->cams) return GS_ERR_INVALID_ARG;
  if (!p->has_fov) return GS_ERR_INVALID_ARG;
  p->last_fov = 1;
  return cuda_status(launch_render(p, ws, true, bg, rgb, T_final, last, stats, stream));
}

gs_status gs_render_backward(gs_plan *p, void *ws, const float *dL_drgb, const float *T_final,
                             const int32_t *last, const float bg[3], float *d_means,
                             float *d_scales, float *d_quats, float *d_opac, float *d_sh,
                             float *d_opac_lv, float *d_dc_lv, cudaStream_t stream) {
  if (!plan_ok(p) || !ws || !dL_drgb || !T_final || !last || !bg || !p->cams) return GS_ERR_INVALID_ARG;
  if (!(p->flags & GS_FLAG_BACKWARD)) return GS_ERR_INVALID_ARG;
  if (p->n > 0 && (!d_means || !d_scales || !d_quats || !d_opac || !d_sh)) return GS_ERR_INVALID_ARG;
  if (p->last_fov && p->fov_mv && ((p->fov.opacity_lv && !d_opac_lv) || (p->fov.dc_lv && !d_dc_lv)))
    return GS_ERR_INVALID_ARG;
  return cuda_status(launch_backward(p, ws, dL_drgb, T_final, last, bg, d_means, d_scales,
                                     d_quats, d_opac, d_sh, d_opac_lv, d_dc_lv, stream));
}

gs_status gs_get_error(const gs_plan *p, const void *ws, cudaStream_t stream, gs_counters *out) {
  if (!plan_ok(p) || !ws) return GS_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return GS_ERR_CUDA;
  Hdr h;
  if (cudaMemcpy(&h, static_cast<const char *>(ws) + p->off[R_HDR], sizeof(Hdr),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return GS_ERR_CUDA;
  if (out) {
    out->status = h.status;
    out->reserved = 0;
    out->n_visible = h.n_visible;
    out->n_pairs = h.n_pairs;
    out->n_nonfinite = h.n_nonfinite;
    out->n_evals = h.n_evals;
    out->n_blends = h.n_blends;
  }
  return (gs_status)h.status;
}

gs_status gs_clear_error(const gs_plan *p, void *ws, cudaStream_t stream) {
  if (!plan_ok(p) || !ws) return GS_ERR_INVALID_ARG;
  return cuda_status(cudaMemsetAsync(region<Hdr>(p, ws, R_HDR), 0, sizeof(uint32_t), stream));
}

gs_status gs_sorted_pairs(const gs_plan *p, const void *ws, cudaStream_t stream,
                          const uint32_t **pair_tile, const uint32_t **pair_item) {
  if (!plan_ok(p) || !ws || !pair_tile || !pair_item) return GS_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return GS_ERR_CUDA;
  Hdr h;
  if (cudaMemcpy(&h, static_cast<const char *>(ws) + p->off[R_HDR], sizeof(Hdr),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return GS_ERR_CUDA;
  const char *b = static_cast<const char *>(ws);
  *pair_tile = reinterpret_cast<const uint32_t *>(b + p->off[h.sel_pair ? R_PKEY_B : R_PKEY_A]);
  *pair_item = reinterpret_cast<const uint32_t *>(b + p->off[h.sel_pair ? R_PVAL_B : R_PVAL_A]);
  return GS_OK;
}

}  // extern "C"
