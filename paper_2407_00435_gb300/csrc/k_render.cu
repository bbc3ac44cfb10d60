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

// Records of one batch in shared memory (structure of arrays).
constexpr int kBatch = 256;

// Prefetched global record of one pair (registers).
struct Pre {
  float4 mean, shape, color;
  uint32_t gid;
  int m;
  bool ok;
};

template <bool FOV>
__device__ __forceinline__ void prefetch(const RenderArgs &a, const uint32_t *vals, uint32_t k,
                                         bool ok, Pre &r) {
  r.ok = ok;
  if (!ok) return;
  const uint32_t j = vals[k];
  r.mean = a.rec_mean[j];
  r.shape = a.rec_shape[j];
  r.color = a.rec_color[j];
  r.gid = a.rec_gid[j];
  r.m = FOV ? (int)a.rec_m[j] : 0;
}

// One block per tile, B*B/PX threads, PX pixels per thread (4 rows apart),
// batches of up to kBatch points staged in shared memory.
template <int B, bool FOV, bool MV, bool STATS, int PX>
__global__ void __launch_bounds__(B * B / PX, 1024 / (B * B / PX)) k_render(RenderArgs a) {
  constexpr int NT = B * B / PX;
  constexpr int NB = 2 * NT < kBatch ? 2 * NT : kBatch;   // points per batch
  constexpr int SPT = NB / NT;                           // points staged per thread
  using G = WarpGeom<B, PX>;
  __shared__ float4 s_a[NB], s_b[NB], s_c[NB];
  __shared__ uint32_t s_gid[STATS ? NB : 1];
  __shared__ int s_m[FOV ? NB : 1];
  __shared__ float4 s_lv[MV ? NB : 1][MV ? kMaxLv : 1];
  __shared__ uint32_t s_cnt[STATS ? NB : 1];
  // per-warp ordered lists of the batch slots that can reach the warp
  constexpr int NWS = NT / 32;                           // staging warps
  __shared__ uint16_t s_list[G::kWarps][NB];
  __shared__ uint16_t s_wcnt[G::kWarps][SPT * NWS];
  __shared__ uint16_t s_woff[G::kWarps][SPT * NWS + 1];

  const long long t = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const ViewDev vd = a.views[find_view(a.views, a.V, t)];
  const int local = (int)(t - vd.tile_base);
  const int tx0 = (local % vd.tx) * B, ty0 = (local / vd.tx) * B;
  const int lx = (warp % G::kWx) * 8 + (lane & 7);
  const int ly0 = (warp / G::kWx) * G::kRows + (lane >> 3);
  int x[PX], y[PX], lvl[PX];
  bool inside[PX], in_band[PX];
  float py[PX], wband[PX];
  Acc A[PX], Bq[PX];
  float dom_w[PX];
  uint32_t dom_gid[PX];
  const float px = (float)lx + 0.5f;
#pragma unroll
  for (int k = 0; k < PX; ++k) {
    const int ly = ly0 + 4 * k;
    x[k] = tx0 + lx;
    y[k] = ty0 + ly;
    inside[k] = x[k] < vd.W && y[k] < vd.H;
    py[k] = (float)ly + 0.5f;
    lvl[k] = 1;
    in_band[k] = false;
    wband[k] = 1.0f;
    if (FOV) pixel_level(vd, a.L, a.band, x[k], y[k], lvl[k], in_band[k], wband[k]);
    A[k] = Acc{0.f, 0.f, 0.f, 1.f, -1, !inside[k]};
    Bq[k] = Acc{0.f, 0.f, 0.f, 1.f, -1, !(inside[k] && in_band[k])};
    dom_w[k] = -1.0f;
    dom_gid[k] = 0;
  }
  uint32_t n_blend = 0;
  uint32_t walk_end[PX];                 // list positions walked until the stop
#pragma unroll
  for (int k = 0; k < PX; ++k) walk_end[k] = 0;
  auto all_done_here = [&]() {
    bool d = true;
#pragma unroll
    for (int k = 0; k < PX; ++k) d = d && A[k].done && Bq[k].done;
    return d;
  };

  const uint2 rg = a.ranges[t];
  const uint32_t *vals = *a.sel ? a.pval_b : a.pval_a;
  if (STATS)
    for (int q = tid; q < NB; q += NT) s_cnt[q] = 0;
  Pre pre[SPT];
#pragma unroll
  for (int u = 0; u < SPT; ++u)
    prefetch<FOV>(a, vals, rg.x + tid + u * NT, rg.x + tid + u * NT < rg.y, pre[u]);

  for (uint32_t b = rg.x;; b += NB) {
    const int all_done = __syncthreads_count(all_done_here()) == NT;
    if (STATS && b > rg.x) {
      for (int q = tid; q < NB; q += NT) {
        const uint32_t c = s_cnt[q];
        if (c) {
          atomicAdd(&a.stats[2 * a.n + s_gid[q]], c);
          atomicAdd(&a.stats[a.n + s_gid[q]], 1u);
          s_cnt[q] = 0;
        }
      }
    }
    if (all_done || b >= rg.y) break;
    const uint32_t cnt = min((uint32_t)NB, rg.y - b);
    uint32_t wm[SPT];
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int q = tid + u * NT;
      wm[u] = 0u;
      if (!pre[u].ok) continue;
      const float mx = (pre[u].mean.x - (float)tx0) + pre[u].mean.z;
      const float my = (pre[u].mean.y - (float)ty0) + pre[u].mean.w;
      float Fmax = pre[u].color.w;
      if (MV) {
        const float4 rest = a.rec_rest[vals[b + q]];
        for (int l = 2; l <= a.L; ++l) {
          float F = pre[u].color.w;
          float4 c = pre[u].color;
          if (a.opacity_lv) F = log2f(a.opacity_lv[(long long)(l - 2) * a.n + pre[u].gid]);
          if (a.dc_lv) {
            const float *dc = a.dc_lv + ((long long)(l - 2) * a.n + pre[u].gid) * 3;
            c.x = fmaxf(0.0f, fmaf(kY00, dc[0], rest.x) + kShOffset);
            c.y = fmaxf(0.0f, fmaf(kY00, dc[1], rest.y) + kShOffset);
            c.z = fmaxf(0.0f, fmaf(kY00, dc[2], rest.z) + kShOffset);
          }
          s_lv[q][l - 2] = make_float4(c.x, c.y, c.z, F);
          Fmax = fmaxf(Fmax, F);
        }
      }
      wm[u] = warp_mask_exact<B, PX>(mx, my, pre[u].shape, Fmax);
      float4 ea, eb;
      make_eval(mx, my, pre[u].shape, pre[u].color.w, wm[u], ea, eb);
      s_a[q] = ea;
      s_b[q] = eb;
      s_c[q] = pre[u].color;
      if (STATS) s_gid[q] = pre[u].gid;
      if (FOV) s_m[q] = pre[u].m;
    }
    // ordered compaction of the slots per target warp: ballot prefixes
    // inside each staging warp, then prefix sums over (u, staging warp)
    uint32_t pfx[SPT][G::kWarps];
#pragma unroll
    for (int u = 0; u < SPT; ++u)
#pragma unroll
      for (int w = 0; w < G::kWarps; ++w) {
        const uint32_t bal = __ballot_sync(0xffffffffu, (wm[u] >> w) & 1u);
        pfx[u][w] = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) s_wcnt[w][u * NWS + warp] = (uint16_t)__popc(bal);
      }
    __syncthreads();
    if (tid < G::kWarps) {
      uint32_t run = 0;
      for (int e = 0; e < SPT * NWS; ++e) {
        s_woff[tid][e] = (uint16_t)run;
        run += s_wcnt[tid][e];
      }
      s_woff[tid][SPT * NWS] = (uint16_t)run;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < SPT; ++u)
#pragma unroll
      for (int w = 0; w < G::kWarps; ++w)
        if ((wm[u] >> w) & 1u) s_list[w][s_woff[w][u * NWS + warp] + pfx[u][w]] = (uint16_t)(tid + u * NT);
    __syncthreads();
    // prefetch the next batch while this one is composited
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const uint32_t k = b + NB + tid + u * NT;
      prefetch<FOV>(a, vals, k, k < rg.y, pre[u]);
    }
    if (!all_done_here()) {
      const int nlist = s_woff[warp][SPT * NWS];
      for (int li = 0; li < nlist; ++li) {
        const uint32_t q = s_list[warp][li];
        const float4 sb = s_b[q];
        const float4 sa = s_a[q];
        const int m = FOV ? s_m[q] : 0;
#pragma unroll
        for (int k = 0; k < PX; ++k) {
          float t1, t2;
          const float sq = eval_s(px, py[k], sa, sb, t1, t2);
          // accumulator A: the pixel's own level
          if (!A[k].done && (!FOV || m >= lvl[k])) {
            const bool own = MV && lvl[k] >= 2;
            const float F = own ? s_lv[q][lvl[k] - 2].w : s_c[q].w;
            const float r2 = own ? __fsub_rn(F, kLog2AlphaMin) : sb.z;
            if (sq <= r2) {
              const float al = alpha_of(__fsub_rn(F, sq));
              const float Tn = A[k].T * (1.0f - al);
              if (Tn < kTMin) {
                A[k].done = true;
                walk_end[k] = b + q - rg.x + 1;
              } else {
                const float4 c = own ? s_lv[q][lvl[k] - 2] : s_c[q];
                const float w = al * A[k].T;
                A[k].r = fmaf(w, c.x, A[k].r);
                A[k].g = fmaf(w, c.y, A[k].g);
                A[k].b = fmaf(w, c.z, A[k].b);
                A[k].T = Tn;
                A[k].last = (int)(b + q - rg.x);
                if (STATS) {
                  ++n_blend;
                  atomicAdd(&s_cnt[q], 1u);
                  if (w > dom_w[k]) { dom_w[k] = w; dom_gid[k] = s_gid[q]; }
                }
              }
            }
          }
          // accumulator B: the better level inside a blend band
          if (FOV && !Bq[k].done && m >= lvl[k] - 1) {
            const bool own = MV && lvl[k] >= 3;
            const float F = own ? s_lv[q][lvl[k] - 3].w : s_c[q].w;
            const float r2 = own ? __fsub_rn(F, kLog2AlphaMin) : sb.z;
            if (sq <= r2) {
              const float al = alpha_of(__fsub_rn(F, sq));
              const float Tn = Bq[k].T * (1.0f - al);
              if (Tn < kTMin) {
                Bq[k].done = true;
              } else {
                const float4 c = own ? s_lv[q][lvl[k] - 3] : s_c[q];
                const float w = al * Bq[k].T;
                Bq[k].r = fmaf(w, c.x, Bq[k].r);
                Bq[k].g = fmaf(w, c.y, Bq[k].g);
                Bq[k].b = fmaf(w, c.z, Bq[k].b);
                Bq[k].T = Tn;
                Bq[k].last = (int)(b + q - rg.x);
              }
            }
          }
        }
        if (all_done_here()) break;
      }
    }
  }
  if (STATS) {
    // block totals of list positions walked until the stop (the same count
    // with or without culling) and of blends (accumulator A)
    unsigned long long e = 0, bl2 = n_blend;
#pragma unroll
    for (int k = 0; k < PX; ++k)
      if (inside[k]) e += (A[k].done && walk_end[k] > 0) ? walk_end[k] : (rg.y - rg.x);
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      bl2 += __shfl_xor_sync(0xffffffffu, bl2, o);
    }
    if (lane == 0) {
      atomicAdd(a.n_evals, e);
      atomicAdd(a.n_blends, bl2);
    }
  }
#pragma unroll
  for (int k = 0; k < PX; ++k) {
    if (!inside[k]) continue;
    const long long pix = vd.pix_base + (long long)y[k] * vd.W + x[k];
    float r = fmaf(A[k].T, a.bg0, A[k].r), g = fmaf(A[k].T, a.bg1, A[k].g),
          bl = fmaf(A[k].T, a.bg2, A[k].b);
    if (FOV) {
      if (in_band[k]) {
        const float rb = fmaf(Bq[k].T, a.bg0, Bq[k].r), gb = fmaf(Bq[k].T, a.bg1, Bq[k].g),
                    bb = fmaf(Bq[k].T, a.bg2, Bq[k].b);
        r = fmaf(wband[k], r - rb, rb);
        g = fmaf(wband[k], g - gb, gb);
        bl = fmaf(wband[k], bl - bb, bb);
      }
      a.T[2 * pix] = A[k].T;
      a.T[2 * pix + 1] = in_band[k] ? Bq[k].T : 1.0f;
      a.last[2 * pix] = A[k].last;
      a.last[2 * pix + 1] = in_band[k] ? Bq[k].last : -1;
    } else {
      a.T[pix] = A[k].T;
      a.last[pix] = A[k].last;
    }
    a.rgb[3 * pix] = r;
    a.rgb[3 * pix + 1] = g;
    a.rgb[3 * pix + 2] = bl;
    if (STATS && A[k].last >= 0) atomicAdd(&a.stats[3 * a.n + dom_gid[k]], 1u);
  }
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
  // plain views: two pixels per thread; foveated: one (two accumulators)
  constexpr int PX = FOV ? 1 : 2;
  k_render<B, FOV, MV, STATS, PX><<<(unsigned)tiles, B * B / PX, 0, s>>>(a);
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
                                           region<uint32_t>(p, ws, R_REC_GID), &hdr->n_items,
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
