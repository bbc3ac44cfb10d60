// gs_internal.cuh -- shared declarations of the CUDA path (not part of the
// public ABI).  Workspace layout, the host-side plan, device-side view table
// and the launchers each translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gs {

// Readings of the constants that the paper defers to the 3DGS paper
// (Sec. 2.1, after Eq. 1).  Kept in one place.
constexpr float kLowpass = 0.3f;          // px^2 added to the 2D covariance
constexpr float kAlphaMax = 0.99f;        // alpha clamp
constexpr float kTMin = 1e-4f;            // stop before T would drop below
constexpr float kClampFov = 1.3f;         // J uses x/z clamped to 1.3 tan(fov/2)
constexpr float kShOffset = 0.5f;         // colour = max(0, SH.Y + 0.5)
// log2(1/255): alpha >= 1/255  <=>  log2(alpha) >= kLog2AlphaMin
constexpr float kLog2AlphaMin = -7.99435343685886f;
// sqrt(0.5 * log2(e)): whitened coordinates t with -(t1^2+t2^2) = log2 of
// exp(-1/2 d^T Q d)
constexpr float kWhiten = 0.84932180028801904f;

constexpr int kMaxViews = 4096;
// selective multi-versioning (per-level opacity / SH DC) holds levels 2..4
constexpr int kMvMaxLevels = 4;

// --------------------------------------------------------------------------
// workspace regions
// --------------------------------------------------------------------------
enum Region : int {
  R_HDR = 0,
  R_VIEWS,
  R_TILE_LEVEL,
  R_LEVEL_ROWS,  // u32 per (tile row, level m): columns whose tile level <= m
                 //   (first | last << 16; first > last when none) [foveated]
  R_REC_MEAN,    // float4 (mx_hi, my_hi, mx_lo, my_lo)
  R_REC_SHAPE,   // float4 whitening rows (w1x, w1y, w2x, w2y)
  R_REC_COLOR,   // float4 (r, g, b, log2 opacity)
  R_REC_REST,    // float4 (view-dependent colour part r, g, b, -) [foveated]
  R_REC_DEPTH,   // u32 float bits of camera z
  R_REC_COUNT,   // u32 kept tile pairs
  R_REC_RECT,    // uint2 packed tile rect (x0 | x1 << 16, y0 | y1 << 16)
  R_REC_GID,     // u32 point index (item slot j = i * V + v)
  R_REC_VIEW,    // u32 view index
  R_REC_M,       // u8 quality bound (foveated)
  R_REC_SUPP,    // float4 tight support (keyed u, v, covariance a, b) [tight]
  R_REC_SUPP2,   // float2 tight support (covariance c, tau) [tight]
  R_REC_EMIT,    // 2 x uint4 emit record per item slot: (corner tile, width | rows << 16,
                 //   tiles per row, count), row intervals of rectangles of <= 8 rows
  R_REC_CBIG,    // u32 count | (item goes to the large-item emit) << 31, visible slots
  R_DKEY_A, R_DKEY_B, R_DVAL_A, R_DVAL_B,   // depth sort ping-pong (M)
  R_OFFSETS,     // u32 exclusive pair offsets in depth order (M)
  R_PKEY_A, R_PKEY_B, R_PVAL_A, R_PVAL_B,   // pair sort ping-pong (K)
  R_BIGQ,        // u32 items with many tiles, expanded by a separate kernel (M)
  R_RANGES,      // uint2 per tile
  R_WORK,        // uint2 chunk slots of the chunked render: (tile, chunk index)
  R_CHUNK_TILE,  // uint4 per tile: (first chunk slot or none, chunks finished,
                 //   first chunk that stopped every pixel, -)
  R_CHUNK_PART,  // float4 per (slot, accumulator, pixel): partial (r, g, b, T)
  R_CHUNK_LAST,  // i32 per (slot, accumulator, pixel): partial last position
  R_BSUM,        // u32 [G][256] per-block digit counts of a sort pass, then
                 //   u64 [G] per-block sums of the pair-offset scan
  R_GRAD_ITEM,   // float per item gradient scratch (backward)
  R_GRAD_LV,     // float per (level, item) gradient scratch (backward, foveated)
  R_COUNT_
};

// Header at the start of the workspace (device).
struct Hdr {
  uint32_t status;
  uint32_t pad0;
  unsigned long long n_visible;   // M: visible (view, point) items
  uint32_t depth_max, depth_nmin;  // largest visible depth key, complement of the smallest
  unsigned long long n_items;     // item slots N * V (visible or not)
  unsigned long long n_pairs;     // K (raw)
  unsigned long long n_nonfinite;
  unsigned long long n_evals;     // (pixel, point) evaluations of the last stats render
  unsigned long long n_blends;    // blends of the last stats render
  uint32_t sel_depth;             // buffer holding the sorted depth order (0 = A)
  uint32_t sel_pair;              // buffer holding the sorted pairs (0 = A)
  uint32_t skip[8];               // per-pass "digit constant" flags
  uint32_t big_count;             // items queued for the large-item emit
  uint32_t pad2;
  uint32_t hist[2][4][256];       // digit histograms: [sort][pass][digit]
  unsigned long long queue;       // next work item of the chunked render
  uint32_t n_slots;               // chunk slots requested by the chunk plan
  uint32_t pad1;
  unsigned long long aux_n;       // key count of a sort outside the frame (pruning)
  unsigned long long aux_out;     // result count of such a pass (compaction)
};

// Per-view constants, computed on the device from the cameras.
struct ViewDev {
  int32_t W, H, tx, ty;
  long long tile_base, pix_base;
  float ccx, ccy, ccz;   // camera centre in world coordinates
  float limx, limy;      // clamp of x/z, y/z used by J
  int32_t fov;           // 1 = foveated
  float gx, gy;          // gaze pixel
  float R[GS_MAX_LEVELS - 1];   // ring radii (px), fy * ring_tan
  int32_t row_base;      // tile rows of the views before this one
};

constexpr int kSpinLimit = 1 << 20;   // bounded waits (about a second), then GS_ERR_TIMEOUT

constexpr int kSortThreads = 256;                     // upsweep / histogram blocks
constexpr int kDownThreads = 512;                     // downsweep blocks
constexpr int kDownItems = 8;                         // keys per downsweep thread
constexpr int kSortPart = kDownThreads * kDownItems;  // 4096 keys per partition
constexpr int kSortBlocksPerSm = 8;   // most sort blocks resident per SM (sizes the block table)
constexpr int kSortMaxBlocks = 1024;  // grid cap of the sort's downsweep
constexpr int kSortSub = 4;           // upsweep sub-ranges per downsweep block
constexpr int kProjThreads = 64;

}  // namespace gs

// Host-side plan (what gs_plan_size() measures).
struct gs_plan {
  uint64_t magic;
  int64_t n;
  int32_t sh_degree, V, tile, chunk;
  uint32_t flags;
  int32_t num_sms;
  int64_t tiles_total, pixels_total, rows_total;
  int64_t max_visible, max_pairs;
  int32_t tile_bits;
  int32_t radix_bits;     // requested digit width of the pair sort (0 = balanced)
  int64_t chunk_cap;      // chunk slots of the chunked render (0 = whole tiles only)
  int32_t sort_blocks;    // rows of the sort's block table (grid upper bound)
  int32_t wait_spins;     // gs_config.wait_spins (projection staging waits)
  int32_t last_fov;       // last render was foveated
  size_t off[gs::R_COUNT_];
  size_t bytes[gs::R_COUNT_];
  size_t ws_bytes;
  // recorded by gs_project
  gs_scene scene;
  const gs_camera *cams;
  int32_t has_fov;
  int32_t fov_mv;         // per-level opacity/DC present
  gs_fov fov;
  int32_t max_w, max_h;
};

namespace gs {

template <typename T>
inline T *region(const gs_plan *p, void *ws, int r) {
  return reinterpret_cast<T *>(static_cast<char *>(ws) + p->off[r]);
}

// ---- launchers (each returns cudaGetLastError()) ------------------------
cudaError_t launch_views(const gs_plan *p, void *ws, cudaStream_t s);
cudaError_t launch_tile_levels(const gs_plan *p, void *ws, cudaStream_t s);
cudaError_t launch_project(const gs_plan *p, void *ws, cudaStream_t s);
// Tile pairs of every visible item (reads the projection's records; run by
// gs_bin_sort beside the depth sort, which does not need them)
cudaError_t launch_count_pairs(const gs_plan *p, void *ws, cudaStream_t s);
cudaError_t launch_bin_sort(const gs_plan *p, void *ws, cudaStream_t s);
cudaError_t launch_render(const gs_plan *p, void *ws, bool fov, const float bg[3],
                          float *rgb, float *T, int32_t *last, uint32_t *stats,
                          cudaStream_t s);
// Stable sort of n uint32 keys with their indices in the plan's depth-sort
// buffers (n <= max_visible); the sorted indices end in R_DVAL_A.
cudaError_t launch_sort_indices(const gs_plan *p, void *ws, const uint32_t *keys, long long n,
                                cudaStream_t s);
cudaError_t launch_backward(const gs_plan *p, void *ws, const float *dL, const float *T,
                            const int32_t *last, const float bg[3], float *d_means,
                            float *d_scales, float *d_quats, float *d_opac, float *d_sh,
                            float *d_opac_lv, float *d_dc_lv, cudaStream_t s);

// device helpers shared by several kernels
__device__ __forceinline__ void set_status(uint32_t *status, uint32_t code) {
  atomicCAS(status, 0u, code);
}

}  // namespace gs
