// k_render.cu -- Rasterization stage (Sec. 2.1, Eq. 1a) for plain and
// foveated views (Sec. 4.1 "Main Pipeline", Sec. 4.2 subsetting and
// multi-versioning), plus the per-point cost statistics of Sec. 3.2.
//
// One block per 16x16 (or 8x8) tile, one pixel per thread.  The tile's
// sorted list is consumed in batches of one point per thread: each thread
// gathers one record into shared memory (2D mean made tile-local from its
// compensated hi/lo form), then every pixel walks the batch front to back.
// A block leaves as soon as every pixel has stopped (block-wide vote).
//
// Per pixel and point: t = W (p - mu) with W the whitened inverse square
// root of the 2D covariance scaled by sqrt(log2(e)/2), so that
//   log2(alpha) = log2(o) - |t|^2,
// alpha floor 1/255 tested on the exponent, clamp 0.99, stop before the
// point that would take T below 1e-4.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_internal.cuh"
#include "raster.cuh"

namespace gs {

constexpr float kY00 = 0.28209479177387814f;   // degree-0 real SH

struct RenderArgs {
  const ViewDev *views;
  int V;
  long long n;
  const uint2 *ranges;
  const uint32_t *pval_a, *pval_b;
  const uint32_t *sel;
  const float4 *rec_mean, *rec_shape, *rec_color, *rec_rest;
  const uint32_t *rec_gid;
  const uint8_t *rec_m;
  int L;
  float band;
  const float *opacity_lv, *dc_lv;
  float bg0, bg1, bg2;
  float *rgb;
  float *T;
  int32_t *last;
  uint32_t *stats;   // (4, N) or null
  unsigned long long *n_evals, *n_blends;
};

struct Acc {
  float r, g, b, T;
  int last;
  bool done;
};

constexpr int kMaxLv = kMvMaxLevels - 1;

template <int B, bool FOV, bool MV, bool STATS>
__global__ void __launch_bounds__(B * B) k_render(RenderArgs a) {
  constexpr int NT = B * B;
  __shared__ float2 s_mean[NT];
  __shared__ float4 s_shape[NT];
  __shared__ float4 s_col[NT];
  __shared__ uint32_t s_gid[NT];
  __shared__ int s_m[FOV ? NT : 1];
  __shared__ float4 s_lv[MV ? NT : 1][MV ? kMaxLv : 1];
  __shared__ uint32_t s_cnt[STATS ? NT : 1];

  const long long t = blockIdx.x;
  const int tid = threadIdx.x;
  const ViewDev vd = a.views[find_view(a.views, a.V, t)];
  const int local = (int)(t - vd.tile_base);
  const int tx0 = (local % vd.tx) * B, ty0 = (local / vd.tx) * B;
  const int lx = tid % B, ly = tid / B;
  const int x = tx0 + lx, y = ty0 + ly;
  const bool inside = x < vd.W && y < vd.H;
  const float px = (float)lx + 0.5f, py = (float)ly + 0.5f;

  // foveation level of this pixel (same FP32 expressions as the filter)
  int lvl = 1;
  bool in_band = false;
  float wband = 1.0f;
  if (FOV) pixel_level(vd, a.L, a.band, x, y, lvl, in_band, wband);
  Acc A = {0.f, 0.f, 0.f, 1.f, -1, !inside};
  Acc Bq = {0.f, 0.f, 0.f, 1.f, -1, !(inside && in_band)};
  float dom_w = -1.0f;
  uint32_t dom_gid = 0;
  uint32_t n_eval = 0, n_blend = 0;

  const uint2 rg = a.ranges[t];
  const uint32_t *vals = *a.sel ? a.pval_b : a.pval_a;
  if (STATS) s_cnt[tid] = 0;

  for (uint32_t b = rg.x;; b += NT) {
    const int all_done = __syncthreads_count(A.done && Bq.done) == NT;
    if (STATS && b > rg.x) {
      uint32_t c = s_cnt[tid];
      if (c) {
        atomicAdd(&a.stats[2 * a.n + s_gid[tid]], c);
        atomicAdd(&a.stats[a.n + s_gid[tid]], 1u);
        s_cnt[tid] = 0;
      }
    }
    if (all_done || b >= rg.y) break;
    const uint32_t cnt = min((uint32_t)NT, rg.y - b);
    if ((uint32_t)tid < cnt) {
      const uint32_t j = vals[b + tid];
      const float4 mean = a.rec_mean[j];
      s_mean[tid] = make_float2((mean.x - (float)tx0) + mean.z, (mean.y - (float)ty0) + mean.w);
      s_shape[tid] = a.rec_shape[j];
      const float4 col = a.rec_color[j];
      s_col[tid] = col;
      const uint32_t gid = a.rec_gid[j];
      s_gid[tid] = gid;
      if (FOV) s_m[tid] = a.rec_m[j];
      if (MV) {
        const float4 rest = a.rec_rest[j];
        for (int l = 2; l <= a.L; ++l) {
          float F = col.w;
          float4 c = col;
          if (a.opacity_lv) F = log2f(a.opacity_lv[(long long)(l - 2) * a.n + gid]);
          if (a.dc_lv) {
            const float *dc = a.dc_lv + ((long long)(l - 2) * a.n + gid) * 3;
            c.x = fmaxf(0.0f, fmaf(kY00, dc[0], rest.x) + kShOffset);
            c.y = fmaxf(0.0f, fmaf(kY00, dc[1], rest.y) + kShOffset);
            c.z = fmaxf(0.0f, fmaf(kY00, dc[2], rest.z) + kShOffset);
          }
          s_lv[tid][l - 2] = make_float4(c.x, c.y, c.z, F);
        }
      }
    }
    __syncthreads();
    if (!(A.done && Bq.done)) {
      for (uint32_t q = 0; q < cnt; ++q) {
        const float2 mu = s_mean[q];
        const float4 sh = s_shape[q];
        float dx, dy, t1, t2;
        const float g = log2_alpha(px, py, mu, sh, 0.0f, dx, dy, t1, t2);
        const int m = FOV ? s_m[q] : 0;
        // accumulator A: the pixel's own level
        if (!A.done && (!FOV || m >= lvl)) {
          const float4 c = (MV && lvl >= 2) ? s_lv[q][lvl - 2] : s_col[q];
          const float p = __fadd_rn(g, c.w);
          if (STATS) ++n_eval;
          if (p >= kLog2AlphaMin) {
            const float al = alpha_of(p);
            const float Tn = A.T * (1.0f - al);
            if (Tn < kTMin) {
              A.done = true;
            } else {
              const float w = al * A.T;
              A.r = fmaf(w, c.x, A.r);
              A.g = fmaf(w, c.y, A.g);
              A.b = fmaf(w, c.z, A.b);
              A.T = Tn;
              A.last = (int)(b + q - rg.x);
              if (STATS) {
                ++n_blend;
                atomicAdd(&s_cnt[q], 1u);
                if (w > dom_w) { dom_w = w; dom_gid = s_gid[q]; }
              }
            }
          }
        }
        // accumulator B: the better level inside a blend band
        if (FOV && !Bq.done && m >= lvl - 1) {
          const float4 c = (MV && lvl >= 3) ? s_lv[q][lvl - 3] : s_col[q];
          const float p = __fadd_rn(g, c.w);
          if (p >= kLog2AlphaMin) {
            const float al = alpha_of(p);
            const float Tn = Bq.T * (1.0f - al);
            if (Tn < kTMin) {
              Bq.done = true;
            } else {
              const float w = al * Bq.T;
              Bq.r = fmaf(w, c.x, Bq.r);
              Bq.g = fmaf(w, c.y, Bq.g);
              Bq.b = fmaf(w, c.z, Bq.b);
              Bq.T = Tn;
              Bq.last = (int)(b + q - rg.x);
            }
          }
        }
        if (A.done && Bq.done) break;
      }
    }
  }
  if (STATS) {
    // block totals of evaluations and blends (accumulator A)
    unsigned long long e = n_eval, bl2 = n_blend;
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      bl2 += __shfl_xor_sync(0xffffffffu, bl2, o);
    }
    if ((tid & 31) == 0) {
      atomicAdd(a.n_evals, e);
      atomicAdd(a.n_blends, bl2);
    }
  }
  if (!inside) return;
  const long long pix = vd.pix_base + (long long)y * vd.W + x;
  float r = fmaf(A.T, a.bg0, A.r), g = fmaf(A.T, a.bg1, A.g), bl = fmaf(A.T, a.bg2, A.b);
  if (FOV) {
    if (in_band) {
      const float rb = fmaf(Bq.T, a.bg0, Bq.r), gb = fmaf(Bq.T, a.bg1, Bq.g),
                  bb = fmaf(Bq.T, a.bg2, Bq.b);
      r = fmaf(wband, r - rb, rb);
      g = fmaf(wband, g - gb, gb);
      bl = fmaf(wband, bl - bb, bb);
    }
    a.T[2 * pix] = A.T;
    a.T[2 * pix + 1] = in_band ? Bq.T : 1.0f;
    a.last[2 * pix] = A.last;
    a.last[2 * pix + 1] = in_band ? Bq.last : -1;
  } else {
    a.T[pix] = A.T;
    a.last[pix] = A.last;
  }
  a.rgb[3 * pix] = r;
  a.rgb[3 * pix + 1] = g;
  a.rgb[3 * pix + 2] = bl;
  if (STATS && A.last >= 0) atomicAdd(&a.stats[3 * a.n + dom_gid], 1u);
}

// tiles_touched (Comp_i) from the per-item pair counts
__global__ void k_tiles_touched(const uint32_t *count, const uint32_t *gid,
                                const unsigned long long *n_items, long long cap,
                                uint32_t *touched) {
  unsigned long long nn = *n_items;
  const long long n = (long long)nn > cap ? cap : (long long)nn;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    uint32_t c = count[j];
    if (c) atomicAdd(&touched[gid[j]], c);
  }
}

template <int B, bool FOV, bool MV, bool STATS>
static void launch_t(const RenderArgs &a, long long tiles, cudaStream_t s) {
  k_render<B, FOV, MV, STATS><<<(unsigned)tiles, B * B, 0, s>>>(a);
}

template <int B>
static void launch_b(const RenderArgs &a, bool fov, bool mv, bool stats, long long tiles,
                     cudaStream_t s) {
  if (!fov) {
    if (stats) launch_t<B, false, false, true>(a, tiles, s);
    else launch_t<B, false, false, false>(a, tiles, s);
  } else if (!mv) {
    if (stats) launch_t<B, true, false, true>(a, tiles, s);
    else launch_t<B, true, false, false>(a, tiles, s);
  } else {
    if (stats) launch_t<B, true, true, true>(a, tiles, s);
    else launch_t<B, true, true, false>(a, tiles, s);
  }
}

cudaError_t launch_render(const gs_plan *p, void *ws, bool fov, const float bg[3], float *rgb,
                          float *T, int32_t *last, uint32_t *stats, cudaStream_t s) {
  Hdr *hdr = region<Hdr>(p, ws, R_HDR);
  if (stats) {
    cudaError_t e = cudaMemsetAsync(stats, 0, sizeof(uint32_t) * 4 * (size_t)p->n, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&hdr->n_evals, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (p->n > 0)
      k_tiles_touched<<<1024, 256, 0, s>>>(region<uint32_t>(p, ws, R_REC_COUNT),
                                           region<uint32_t>(p, ws, R_REC_GID), &hdr->n_visible,
                                           p->max_visible, stats);
  }
  if (p->tiles_total == 0) return cudaGetLastError();
  RenderArgs a = {};
  a.views = region<ViewDev>(p, ws, R_VIEWS);
  a.V = p->V;
  a.n = p->n;
  a.ranges = region<uint2>(p, ws, R_RANGES);
  a.pval_a = region<uint32_t>(p, ws, R_PVAL_A);
  a.pval_b = region<uint32_t>(p, ws, R_PVAL_B);
  a.sel = &hdr->sel_pair;
  a.rec_mean = region<float4>(p, ws, R_REC_MEAN);
  a.rec_shape = region<float4>(p, ws, R_REC_SHAPE);
  a.rec_color = region<float4>(p, ws, R_REC_COLOR);
  a.rec_rest = p->bytes[R_REC_REST] ? region<float4>(p, ws, R_REC_REST) : nullptr;
  a.rec_gid = region<uint32_t>(p, ws, R_REC_GID);
  a.rec_m = p->bytes[R_REC_M] ? region<uint8_t>(p, ws, R_REC_M) : nullptr;
  a.L = fov ? p->fov.n_levels : 1;
  a.band = fov ? p->fov.band_px : 0.0f;
  a.opacity_lv = fov ? p->fov.opacity_lv : nullptr;
  a.dc_lv = fov ? p->fov.dc_lv : nullptr;
  a.bg0 = bg[0];
  a.bg1 = bg[1];
  a.bg2 = bg[2];
  a.rgb = rgb;
  a.T = T;
  a.last = last;
  a.stats = stats;
  a.n_evals = &hdr->n_evals;
  a.n_blends = &hdr->n_blends;
  const bool mv = fov && p->fov_mv;
  if (p->tile == 16) launch_b<16>(a, fov, mv, stats != nullptr, p->tiles_total, s);
  else launch_b<8>(a, fov, mv, stats != nullptr, p->tiles_total, s);
  return cudaGetLastError();
}

}  // namespace gs
