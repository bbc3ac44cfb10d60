// k_render.cu -- Rasterization stage (Sec. 2.1, Eq. 1a) for plain and
// foveated views (Sec. 4.1 "Main Pipeline", Sec. 4.2 subsetting and
// multi-versioning), plus the per-point cost statistics of Sec. 3.2.
//
// One block per 16x16 (or 8x8) tile, two pixels per thread 4 rows apart
// (one for foveated renders with per-level parameters or statistics).  The
// tile's sorted list is consumed in batches: each thread gathers records into
// shared memory (2D mean made tile-local from its compensated hi/lo form),
// ordered per-warp lists of the points that can reach each warp are built,
// then every warp walks its list front to back.  A block leaves as soon as
// every pixel has stopped (block-wide vote).
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
  int mmfr;                      // a separate model per level (GS_FLAG_MULTI_MODEL)
  const float *opacity_lv, *dc_lv;
  float bg0, bg1, bg2;
  float *rgb;
  float *T;
  int32_t *last;
  uint32_t *stats;   // (4, N) or null
  unsigned long long *n_evals, *n_blends;
  // heavy-tile chunking (persistent work queue)
  int chunk;                     // points per chunk
  long long tiles;
  const uint2 *chunk_list;       // per slot: (tile, chunk index); y = kNoChunk: unused
  uint4 *chunk_tile;             // per tile: (first slot or kNoChunk, chunks finished,
                                 //   first chunk whose pixels all stopped, -)
  float4 *part_ct;               // per (slot, accumulator, pixel): (r, g, b, +-T)
  int32_t *part_last;            // per (slot, accumulator, pixel): last blended position
  unsigned long long ch_cap;     // chunk slots held by the workspace
  const uint32_t *n_slots;       // chunk slots requested by k_chunk_plan
  unsigned long long *queue;     // next work item
};

constexpr uint32_t kNoChunk = 0xffffffffu;

struct Acc {
  float r, g, b, T;
  int last;
  bool done;
};

constexpr int kMaxLv = kMvMaxLevels - 1;

// Records of one batch in shared memory (structure of arrays).
constexpr int kBatch = 128;   // points per batch: one per thread (measured faster than 256)

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

// Block-uniform description of the current work item, kept in shared
// memory so that it does not occupy registers across the walks.
struct ItemSm {
  long long t;                       // tile
  unsigned long long slot, first;    // this chunk's slot, the tile's first slot
  uint32_t nc, cc, c;                // chunks of the tile (0: whole), chunk being merged,
                                     //   this item's chunk
  uint32_t begin, end, origin;       // walked range, first pair of the tile
  int vidx, tx0, ty0;                // view, tile origin in pixels
  int merging;
};

// Shared memory of one render block: the records of one batch (structure
// of arrays) and the per-warp ordered lists of the batch slots that can
// reach each warp.
template <int B, bool FOV, bool MV, bool STATS, int PX>
struct RSmem {
  static constexpr int NT = B * B / PX;                   // threads
  static constexpr int NB = 2 * NT < kBatch ? 2 * NT : (NT > kBatch ? NT : kBatch);
  static constexpr int SPT = NB / NT;                     // points staged per thread
  static constexpr int NWS = NT / 32;                     // staging warps
  static constexpr int NW = WarpGeom<B, PX>::kWarps;
  float4 a[NB], b[NB], c[NB];
  uint32_t gid[STATS ? NB : 1];
  int m[FOV ? NB : 1];
  float4 lv[MV ? NB : 1][MV ? kMaxLv : 1];
  uint32_t cnt[STATS ? NB : 1];
  uint16_t list[NW][NB];
  uint16_t wcnt[NW][SPT * NWS];
  uint16_t woff[NW][SPT * NWS + 1];
  // per warp: the lowest level its pixels need | the highest own level << 8
  // (a point whose m no pixel of the warp can use is left out of its list)
  uint16_t wlv[FOV ? NW : 1];
  unsigned long long item;   // work-queue item broadcast
  int flag;                  // last chunk of a tile to arrive
  int abort;                 // an earlier chunk of the tile stopped every pixel
  ItemSm it;
};

// Per-thread pixel state used by the walk (PX pixels 4 rows apart).
template <int PX>
struct Pix {
  float px, py[PX];   // tile-local pixel centre
  int lvl[PX];        // foveation level
};

// Plain views: composites the warp's ordered list of batch slots into the
// thread's PX pixels.  The per-pixel decisions are written as data flow (the
// compiler predicates them instead of branching), every lane takes the
// warp's trip count, and the warp leaves once none of its pixels is live,
// checked every 4 entries.  Decisions and arithmetic are those of the
// generic loop in walk().
template <int PX>
__device__ __forceinline__ void composite_plain(const uint16_t *list, int nlist,
                                                const float4 *ra, const float4 *rb,
                                                const float4 *rc, int base, const Pix<PX> &pp,
                                                Acc (&A)[PX], uint32_t (&walk_end)[PX]) {
  // pixel centres packed twice: the paired FMA operands of eval_s2
  const unsigned long long px2 = f2_pack(pp.px, pp.px);
  unsigned long long py2[PX];
#pragma unroll
  for (int k = 0; k < PX; ++k) py2[k] = f2_pack(pp.py[k], pp.py[k]);
  // unrolled so that the shared-memory loads of later entries are issued
  // above the arithmetic of earlier ones (measured faster than 1, 2, 4 or 6)
#pragma unroll 8
  for (int li = 0; li < nlist; ++li) {
    const int q = list[li];
    const float4 sa = ra[q], sb = rb[q], c = rc[q];
    const int pos = base + q;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
      float t1, t2;
      const float sq = eval_s2(px2, py2[k], sa, sb, t1, t2);
      const float al = alpha_of(__fsub_rn(c.w, sq));
      const float Tn = __fmaf_rn(-al, A[k].T, A[k].T);
      const bool hit = !A[k].done && sq <= sb.z;
      if (hit && !(Tn < kTMin)) {
        const float w = al * A[k].T;
        A[k].r = fmaf(w, c.x, A[k].r);
        A[k].g = fmaf(w, c.y, A[k].g);
        A[k].b = fmaf(w, c.z, A[k].b);
        A[k].T = Tn;
        A[k].last = pos;
      }
      if (hit && Tn < kTMin) {
        A[k].done = true;
        walk_end[k] = pos + 1;
      }
    }
    if ((li & 3) == 3) {
      // leave once no pixel of the warp is still compositing
      bool live = false;
#pragma unroll
      for (int k = 0; k < PX; ++k) live = live || !A[k].done;
      if (!__any_sync(0xffffffffu, live)) break;
    }
  }
}

// Foveated views, warps with no pixel in a blend band: accumulator A only,
// composited as in composite_plain; a point takes part where its level bit
// mask holds the pixel's level.
template <int PX>
__device__ __forceinline__ void composite_fov_a(const uint16_t *list, int nlist,
                                                const float4 *ra, const float4 *rb,
                                                const float4 *rc, const int *rm, int base,
                                                const Pix<PX> &pp, Acc (&A)[PX],
                                                uint32_t (&walk_end)[PX]) {
  const unsigned long long px2 = f2_pack(pp.px, pp.px);
  unsigned long long py2[PX];
  uint32_t bit[PX];
#pragma unroll
  for (int k = 0; k < PX; ++k) {
    py2[k] = f2_pack(pp.py[k], pp.py[k]);
    bit[k] = 1u << (pp.lvl[k] - 1);
  }
#pragma unroll 8
  for (int li = 0; li < nlist; ++li) {
    const int q = list[li];
    const float4 sa = ra[q], sb = rb[q], c = rc[q];
    const uint32_t pm = (uint32_t)rm[q];
    const int pos = base + q;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
      float t1, t2;
      const float sq = eval_s2(px2, py2[k], sa, sb, t1, t2);
      const float al = alpha_of(__fsub_rn(c.w, sq));
      const float Tn = __fmaf_rn(-al, A[k].T, A[k].T);
      const bool hit = !A[k].done && (pm & bit[k]) != 0u && sq <= sb.z;
      if (hit && !(Tn < kTMin)) {
        const float w = al * A[k].T;
        A[k].r = fmaf(w, c.x, A[k].r);
        A[k].g = fmaf(w, c.y, A[k].g);
        A[k].b = fmaf(w, c.z, A[k].b);
        A[k].T = Tn;
        A[k].last = pos;
      }
      if (hit && Tn < kTMin) {
        A[k].done = true;
        walk_end[k] = pos + 1;
      }
    }
    if ((li & 3) == 3) {
      // leave once no pixel of the warp is still compositing
      bool live = false;
#pragma unroll
      for (int k = 0; k < PX; ++k) live = live || !A[k].done;
      if (!__any_sync(0xffffffffu, live)) break;
    }
  }
}

// Foveated views, warps with a pixel in a blend band (no per-level
// parameters, no statistics): both accumulators from one evaluation of the
// quadratic form, the decisions as data flow like composite_plain; a point
// takes part in accumulator A where its level mask holds the pixel's level,
// in B where it holds the level below (0 outside bands).
template <int PX>
__device__ __forceinline__ void composite_fov_ab(const uint16_t *list, int nlist,
                                                 const float4 *ra, const float4 *rb,
                                                 const float4 *rc, const int *rm, int base,
                                                 const Pix<PX> &pp, Acc (&A)[PX], Acc (&Bq)[PX],
                                                 uint32_t (&walk_end)[PX]) {
  const unsigned long long px2 = f2_pack(pp.px, pp.px);
  unsigned long long py2[PX];
  uint32_t bitA[PX], bitB[PX];
#pragma unroll
  for (int k = 0; k < PX; ++k) {
    py2[k] = f2_pack(pp.py[k], pp.py[k]);
    bitA[k] = 1u << (pp.lvl[k] - 1);
    bitB[k] = pp.lvl[k] >= 2 ? 1u << (pp.lvl[k] - 2) : 0u;
  }
#pragma unroll 4
  for (int li = 0; li < nlist; ++li) {
    const int q = list[li];
    const float4 sa = ra[q], sb = rb[q], c = rc[q];
    const uint32_t pm = (uint32_t)rm[q];
    const int pos = base + q;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
      float t1, t2;
      const float sq = eval_s2(px2, py2[k], sa, sb, t1, t2);
      const float al = alpha_of(__fsub_rn(c.w, sq));
      const bool in = sq <= sb.z;
      {
        const float Tn = __fmaf_rn(-al, A[k].T, A[k].T);
        const bool hit = in && !A[k].done && (pm & bitA[k]) != 0u;
        if (hit && !(Tn < kTMin)) {
          const float w = al * A[k].T;
          A[k].r = fmaf(w, c.x, A[k].r);
          A[k].g = fmaf(w, c.y, A[k].g);
          A[k].b = fmaf(w, c.z, A[k].b);
          A[k].T = Tn;
          A[k].last = pos;
        }
        if (hit && Tn < kTMin) {
          A[k].done = true;
          walk_end[k] = pos + 1;
        }
      }
      {
        const float Tn = __fmaf_rn(-al, Bq[k].T, Bq[k].T);
        const bool hit = in && !Bq[k].done && (pm & bitB[k]) != 0u;
        if (hit && !(Tn < kTMin)) {
          const float w = al * Bq[k].T;
          Bq[k].r = fmaf(w, c.x, Bq[k].r);
          Bq[k].g = fmaf(w, c.y, Bq[k].g);
          Bq[k].b = fmaf(w, c.z, Bq[k].b);
          Bq[k].T = Tn;
          Bq[k].last = pos;
        }
        if (hit && Tn < kTMin) Bq[k].done = true;
      }
    }
    if ((li & 3) == 3) {
      bool live = false;
#pragma unroll
      for (int k = 0; k < PX; ++k) live = live || !A[k].done || !Bq[k].done;
      if (!__any_sync(0xffffffffu, live)) break;
    }
  }
}

// Composites the sorted points [begin, end) of a tile front to back into
// every accumulator that is not done.  List positions (`last`) are reported
// relative to `origin`, the first pair of the tile.  Starts and ends with a
// block-wide barrier, so the shared batch buffers can be reused right after.
template <int B, bool FOV, bool MV, bool STATS, int PX>
__device__ __forceinline__ void walk(const RenderArgs &a, RSmem<B, FOV, MV, STATS, PX> &sm,
                                     const uint32_t *vals, int tx0, int ty0, uint32_t begin,
                                     uint32_t end, uint32_t origin, const Pix<PX> &pp,
                                     Acc (&A)[PX], Acc (&Bq)[PX], float (&dom_w)[PX],
                                     uint32_t (&dom_gid)[PX], uint32_t &n_blend,
                                     uint32_t (&walk_end)[PX], const uint32_t *stop_c = nullptr,
                                     uint32_t my_c = 0) {
  using S = RSmem<B, FOV, MV, STATS, PX>;
  constexpr int NT = S::NT, NB = S::NB, SPT = S::SPT, NWS = S::NWS;
  using G = WarpGeom<B, PX>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto all_done_here = [&]() {
    bool d = true;
#pragma unroll
    for (int k = 0; k < PX; ++k) d = d && A[k].done && Bq[k].done;
    return d;
  };
  if (STATS)
    for (int q = tid; q < NB; q += NT) sm.cnt[q] = 0;
  Pre pre[SPT];
#pragma unroll
  for (int u = 0; u < SPT; ++u)
    prefetch<FOV>(a, vals, begin + tid + u * NT, begin + tid + u * NT < end, pre[u]);

  for (uint32_t b = begin;; b += NB) {
    // a chunk stops early once an earlier chunk of its tile has stopped
    // every pixel: the merge never reads what would follow
    if (stop_c && tid == 0 && *(const volatile uint32_t *)stop_c < my_c) sm.abort = 1;
    const int all_done = __syncthreads_count(all_done_here()) == NT;
    if (STATS && b > begin) {
      for (int q = tid; q < NB; q += NT) {
        const uint32_t c = sm.cnt[q];
        if (c) {
          atomicAdd(&a.stats[2 * a.n + sm.gid[q]], c);
          atomicAdd(&a.stats[a.n + sm.gid[q]], 1u);
          sm.cnt[q] = 0;
        }
      }
    }
    if (all_done || b >= end || (stop_c && sm.abort)) break;
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
          sm.lv[q][l - 2] = make_float4(c.x, c.y, c.z, F);
          Fmax = fmaxf(Fmax, F);
        }
      }
      wm[u] = warp_mask_exact<B, PX>(mx, my, pre[u].shape, Fmax);
      if (FOV) {
#pragma unroll
        for (int w = 0; w < G::kWarps; ++w) {
          const int lo = sm.wlv[w] & 0xff, hi = sm.wlv[w] >> 8;
          const int m = pre[u].m;
          if (a.mmfr ? (m < lo || m > hi) : m < lo) wm[u] &= ~(1u << w);
        }
      }
      float4 ea, eb;
      make_eval(mx, my, pre[u].shape, pre[u].color.w, wm[u], ea, eb);
      sm.a[q] = ea;
      sm.b[q] = eb;
      sm.c[q] = pre[u].color;
      if (STATS) sm.gid[q] = pre[u].gid;
      // levels the point takes part in, as a bit mask (bit l - 1: level l):
      // levels 1..m for nested subsets, level m alone with a model per level
      if (FOV) {
        const int m = pre[u].m;
        sm.m[q] = m < 1 ? 0 : (a.mmfr ? (1 << (m - 1)) : (1 << m) - 1);
      }
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
        if (lane == 0) sm.wcnt[w][u * NWS + warp] = (uint16_t)__popc(bal);
      }
    __syncthreads();
    if (tid < G::kWarps) {
      uint32_t run = 0;
      for (int e = 0; e < SPT * NWS; ++e) {
        sm.woff[tid][e] = (uint16_t)run;
        run += sm.wcnt[tid][e];
      }
      sm.woff[tid][SPT * NWS] = (uint16_t)run;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < SPT; ++u)
#pragma unroll
      for (int w = 0; w < G::kWarps; ++w)
        if ((wm[u] >> w) & 1u)
          sm.list[w][sm.woff[w][u * NWS + warp] + pfx[u][w]] = (uint16_t)(tid + u * NT);
    __syncthreads();
    // prefetch the next batch while this one is composited
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const uint32_t k = b + NB + tid + u * NT;
      prefetch<FOV>(a, vals, k, k < end, pre[u]);
    }
    if (!FOV && !STATS) {
      if (__any_sync(0xffffffffu, !all_done_here()))
        composite_plain<PX>(sm.list[warp], sm.woff[warp][SPT * NWS], sm.a, sm.b, sm.c,
                            (int)(b - origin), pp, A, walk_end);
    } else if (FOV && !MV && !STATS &&
               __all_sync(0xffffffffu, [&] {
                 bool nb = true;
#pragma unroll
                 for (int k = 0; k < PX; ++k) nb = nb && Bq[k].done;
                 return nb;
               }())) {
      // no pixel of the warp needs the second accumulator; if every pixel
      // has the same level the warp's list holds exactly the points that
      // level composites (the list excludes the others), so no level test
      if (__any_sync(0xffffffffu, !all_done_here())) {
        const int lo = sm.wlv[warp] & 0xff, hi = sm.wlv[warp] >> 8;
        if (lo == hi)
          composite_plain<PX>(sm.list[warp], sm.woff[warp][SPT * NWS], sm.a, sm.b, sm.c,
                              (int)(b - origin), pp, A, walk_end);
        else
          composite_fov_a<PX>(sm.list[warp], sm.woff[warp][SPT * NWS], sm.a, sm.b, sm.c, sm.m,
                              (int)(b - origin), pp, A, walk_end);
      }
    } else if (FOV && !MV && !STATS) {
      if (__any_sync(0xffffffffu, !all_done_here()))
        composite_fov_ab<PX>(sm.list[warp], sm.woff[warp][SPT * NWS], sm.a, sm.b, sm.c, sm.m,
                             (int)(b - origin), pp, A, Bq, walk_end);
    } else if (__any_sync(0xffffffffu, !all_done_here())) {
      const int nlist = sm.woff[warp][SPT * NWS];
      const unsigned long long px2 = f2_pack(pp.px, pp.px);
      unsigned long long py2[PX];
#pragma unroll
      for (int k = 0; k < PX; ++k) py2[k] = f2_pack(pp.py[k], pp.py[k]);
      // level bits of the two accumulators (own level; one below in a band)
      uint32_t bitA[PX], bitB[PX];
#pragma unroll
      for (int k = 0; k < PX; ++k) {
        bitA[k] = 1u << (pp.lvl[k] - 1);
        bitB[k] = pp.lvl[k] >= 2 ? 1u << (pp.lvl[k] - 2) : 0u;
      }
#pragma unroll 4
      for (int li = 0; li < nlist; ++li) {
        const uint32_t q = sm.list[warp][li];
        const float4 sb = sm.b[q];
        const float4 sa = sm.a[q];
        const uint32_t pm = FOV ? (uint32_t)sm.m[q] : 0u;
#pragma unroll
        for (int k = 0; k < PX; ++k) {
          float t1, t2;
          const float sq = eval_s2(px2, py2[k], sa, sb, t1, t2);
          // accumulator A: the pixel's own level
          if (!A[k].done && (!FOV || (pm & bitA[k]))) {
            const bool own = MV && pp.lvl[k] >= 2;
            const float F = own ? sm.lv[q][pp.lvl[k] - 2].w : sm.c[q].w;
            const float r2 = own ? __fsub_rn(F, kLog2AlphaMin) : sb.z;
            if (sq <= r2) {
              const float al = alpha_of(__fsub_rn(F, sq));
              const float Tn = __fmaf_rn(-al, A[k].T, A[k].T);
              if (Tn < kTMin) {
                A[k].done = true;
                walk_end[k] = b + q - origin + 1;
              } else {
                const float4 c = own ? sm.lv[q][pp.lvl[k] - 2] : sm.c[q];
                const float w = al * A[k].T;
                A[k].r = fmaf(w, c.x, A[k].r);
                A[k].g = fmaf(w, c.y, A[k].g);
                A[k].b = fmaf(w, c.z, A[k].b);
                A[k].T = Tn;
                A[k].last = (int)(b + q - origin);
                if (STATS) {
                  ++n_blend;
                  atomicAdd(&sm.cnt[q], 1u);
                  if (w > dom_w[k]) { dom_w[k] = w; dom_gid[k] = sm.gid[q]; }
                }
              }
            }
          }
          // accumulator B: the better level inside a blend band
          if (FOV && !Bq[k].done && (pm & bitB[k])) {
            const bool own = MV && pp.lvl[k] >= 3;
            const float F = own ? sm.lv[q][pp.lvl[k] - 3].w : sm.c[q].w;
            const float r2 = own ? __fsub_rn(F, kLog2AlphaMin) : sb.z;
            if (sq <= r2) {
              const float al = alpha_of(__fsub_rn(F, sq));
              const float Tn = __fmaf_rn(-al, Bq[k].T, Bq[k].T);
              if (Tn < kTMin) {
                Bq[k].done = true;
              } else {
                const float4 c = own ? sm.lv[q][pp.lvl[k] - 3] : sm.c[q];
                const float w = al * Bq[k].T;
                Bq[k].r = fmaf(w, c.x, Bq[k].r);
                Bq[k].g = fmaf(w, c.y, Bq[k].g);
                Bq[k].b = fmaf(w, c.z, Bq[k].b);
                Bq[k].T = Tn;
                Bq[k].last = (int)(b + q - origin);
              }
            }
          }
        }
        if ((li & 3) == 3 && !__any_sync(0xffffffffu, !all_done_here())) break;
      }
    }
  }
}

// Folds the partial result (C_c, T_c) of chunk c into an accumulator that
// has composited chunks 0..c-1:  (C, T) o (C_c, T_c) = (C + T C_c, T T_c).
// A chunk walked from T = 1 stops when its own T would drop below 1e-4;
// with the incoming T the true stop can only come earlier, so a chunk that
// stopped (T_c stored negated), or whose product crosses 1e-4, has to be
// re-walked from the incoming state: returns true then.  With nothing
// composited before (T == 1) the chunk's own walk is already exact.
__device__ __forceinline__ bool merge_chunk(Acc &X, float4 part, int plast) {
  if (X.done) return false;
  const float Tc = fabsf(part.w);
  const bool stopped = part.w < 0.0f;
  if (X.T == 1.0f) {
    X.r = part.x;
    X.g = part.y;
    X.b = part.z;
    X.T = Tc;
    if (plast >= 0) X.last = plast;
    X.done = stopped;
    return false;
  }
  if (stopped || X.T * Tc < kTMin) return true;
  X.r = fmaf(X.T, part.x, X.r);
  X.g = fmaf(X.T, part.y, X.g);
  X.b = fmaf(X.T, part.z, X.b);
  X.T = X.T * Tc;
  if (plast >= 0) X.last = plast;
  return false;
}

// Image position and foveation of pixel k of this thread in a tile.
template <int B, bool FOV, int PX>
__device__ __forceinline__ void pixel_of(const RenderArgs &a, const ViewDev &vd, int tx0, int ty0,
                                         int k, int &x, int &y, int &lvl, bool &inside,
                                         bool &in_band, float &wband) {
  using G = WarpGeom<B, PX>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  x = tx0 + (warp % G::kWx) * 8 + (lane & 7);
  y = ty0 + (warp / G::kWx) * G::kRows + (lane >> 3) + 4 * k;
  inside = x < vd.W && y < vd.H;
  lvl = 1;
  in_band = false;
  wband = 1.0f;
  if (FOV) pixel_level(vd, a.L, a.band, x, y, lvl, in_band, wband);
}

// One work item: the whole tile t (nc == 0), or chunk c of the nc chunks of
// a heavy tile, whose partial result goes to chunk slot `slot`.  The last
// chunk of a tile to finish merges all of them and writes the pixels.
template <int B, bool FOV, bool MV, bool STATS, int PX, bool CHUNK>
__device__ __forceinline__ void render_item(const RenderArgs &a,
                                            RSmem<B, FOV, MV, STATS, PX> &sm,
                                            const uint32_t *vals, long long t, uint32_t c,
                                            unsigned long long slot, uint32_t nc) {
  using G = WarpGeom<B, PX>;
  constexpr int NACC = FOV ? 2 : 1;
  constexpr size_t BB = (size_t)B * B;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lx = (warp % G::kWx) * 8 + (lane & 7);
  const int ly0 = (warp / G::kWx) * G::kRows + (lane >> 3);
  Pix<PX> pp;
  Acc A[PX], Bq[PX];
  float dom_w[PX];
  uint32_t dom_gid[PX];
  uint32_t inb = 0;                // bits: inside k, in band PX + k
  uint32_t begin, end, origin;
  int tx0, ty0;
  {
    const int vidx = find_view(a.views, a.V, t);
    const ViewDev vd = a.views[vidx];
    const int local = (int)(t - vd.tile_base);
    tx0 = (local % vd.tx) * B;
    ty0 = (local / vd.tx) * B;
    const uint2 rg = a.ranges[t];
    origin = rg.x;
    begin = rg.x;
    end = rg.y;
    if (CHUNK && nc) {
      begin = rg.x + c * (uint32_t)a.chunk;
      end = min(rg.y, begin + (uint32_t)a.chunk);
    }
    pp.px = (float)lx + 0.5f;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
      int x, y;
      bool inside, in_band;
      float wband;
      pixel_of<B, FOV, PX>(a, vd, tx0, ty0, k, x, y, pp.lvl[k], inside, in_band, wband);
      pp.py[k] = (float)(ly0 + 4 * k) + 0.5f;
      inb |= (inside ? 1u : 0u) << k;
      inb |= (inside && in_band ? 1u : 0u) << (PX + k);
      A[k] = Acc{0.f, 0.f, 0.f, 1.f, -1, !inside};
      Bq[k] = Acc{0.f, 0.f, 0.f, 1.f, -1, !(inside && in_band)};
      dom_w[k] = -1.0f;
      dom_gid[k] = 0;
    }
    if (FOV) {
      // the levels this warp's pixels use: own level, and one below in a band
      int lo = 255, hi = 0;
#pragma unroll
      for (int k = 0; k < PX; ++k)
        if ((inb >> k) & 1u) {
          lo = min(lo, pp.lvl[k] - (int)((inb >> (PX + k)) & 1u));
          hi = max(hi, pp.lvl[k]);
        }
      for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      if (lane == 0) sm.wlv[warp] = (uint16_t)(lo | (hi << 8));
    }
    if (CHUNK && tid == 0) {
      sm.abort = 0;
      sm.it.t = t;
      sm.it.slot = slot;
      sm.it.nc = nc;
      sm.it.c = c;
      sm.it.vidx = vidx;
      sm.it.tx0 = tx0;
      sm.it.ty0 = ty0;
      sm.it.origin = origin;
      sm.it.end = rg.y;
      sm.it.merging = 0;
    }
  }
  uint32_t n_blend = 0;
  uint32_t walk_end[PX];                 // list positions walked until the stop
#pragma unroll
  for (int k = 0; k < PX; ++k) walk_end[k] = 0;

  // One walk call site (the loop keeps a single inlined copy): the item's
  // own walk, then, for the last chunk of a heavy tile to finish, the merge
  // with its re-walks of the chunks in which an early stop falls.  Item
  // constants are re-read from shared memory after each walk.
  uint32_t fix = 0, keep = 0;      // per accumulator bits: k (A), PX + k (B)
  const uint32_t *stop_c = (CHUNK && nc && c > 0) ? &a.chunk_tile[t].z : nullptr;
  for (;;) {
    walk<B, FOV, MV, STATS, PX>(a, sm, vals, tx0, ty0, begin, end, origin, pp, A, Bq, dom_w,
                                dom_gid, n_blend, walk_end, stop_c, c);
    stop_c = nullptr;   // re-walks of the merge run to their stop
    if (!CHUNK) break;
    const uint32_t inc = sm.it.nc;
    if (inc == 0) break;
    uint32_t cc;
    if (!sm.it.merging) {
      // partial result of this chunk; T negated where the chunk's walk stopped
      const unsigned long long sl = sm.it.slot;
      const bool aborted = sm.abort;
      bool all_stopped = true;
#pragma unroll
      for (int k = 0; k < PX; ++k) all_stopped = all_stopped && A[k].done && Bq[k].done;
#pragma unroll
      for (int k = 0; k < PX; ++k) {
        if (aborted || !((inb >> k) & 1u)) continue;
        const size_t i = sl * NACC * BB + (size_t)((ly0 + 4 * k) * B + lx);
        a.part_ct[i] = make_float4(A[k].r, A[k].g, A[k].b, A[k].done ? -A[k].T : A[k].T);
        a.part_last[i] = A[k].last;
        if (FOV && ((inb >> (PX + k)) & 1u)) {
          a.part_ct[i + BB] =
              make_float4(Bq[k].r, Bq[k].g, Bq[k].b, Bq[k].done ? -Bq[k].T : Bq[k].T);
          a.part_last[i + BB] = Bq[k].last;
        }
      }
      __threadfence();
      all_stopped = __syncthreads_and(all_stopped) && !aborted;
      if (tid == 0) {
        const long long tt = sm.it.t;
        if (all_stopped) atomicMin(&a.chunk_tile[tt].z, sm.it.c);
        sm.flag = atomicAdd(&a.chunk_tile[tt].y, 1u) == inc - 1;
        sm.it.first = a.chunk_tile[tt].x;
        sm.it.merging = 1;
      }
      __syncthreads();
      if (!sm.flag) return;
      __threadfence();
      // last to arrive: merge the chunks in list order
      cc = 0;
#pragma unroll
      for (int k = 0; k < PX; ++k) {
        A[k] = Acc{0.f, 0.f, 0.f, 1.f, -1, !((inb >> k) & 1u)};
        Bq[k] = Acc{0.f, 0.f, 0.f, 1.f, -1, !((inb >> (PX + k)) & 1u)};
      }
    } else {
      // chunk cc re-walked: accumulators that sat it out resume their state
#pragma unroll
      for (int k = 0; k < PX; ++k) {
        if (!((fix >> k) & 1u)) A[k].done = (keep >> k) & 1u;
        if (!((fix >> (PX + k)) & 1u)) Bq[k].done = (keep >> (PX + k)) & 1u;
      }
      cc = sm.it.cc + 1;
    }
    const unsigned long long fs = sm.it.first;
    bool rewalk = false;
    for (; cc < inc; ++cc) {
      fix = 0;
#pragma unroll
      for (int k = 0; k < PX; ++k) {
        const size_t i = (fs + cc) * NACC * BB + (size_t)((ly0 + 4 * k) * B + lx);
        if (!A[k].done && merge_chunk(A[k], __ldcg(&a.part_ct[i]), __ldcg(&a.part_last[i])))
          fix |= 1u << k;
        if (FOV && !Bq[k].done &&
            merge_chunk(Bq[k], __ldcg(&a.part_ct[i + BB]), __ldcg(&a.part_last[i + BB])))
          fix |= 1u << (PX + k);
      }
      if (__syncthreads_or(fix != 0)) {
        rewalk = true;
        break;
      }
    }
    if (!rewalk) break;
    // re-walk chunk cc for the accumulators whose stop falls inside it
    keep = 0;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
      keep |= (A[k].done ? 1u : 0u) << k;
      keep |= (Bq[k].done ? 1u : 0u) << (PX + k);
      A[k].done = !((fix >> k) & 1u);
      Bq[k].done = !((fix >> (PX + k)) & 1u);
    }
    if (tid == 0) sm.it.cc = cc;
    tx0 = sm.it.tx0;
    ty0 = sm.it.ty0;
    origin = sm.it.origin;
    begin = origin + cc * (uint32_t)a.chunk;
    end = min(sm.it.end, begin + (uint32_t)a.chunk);
  }

  // output
  const ViewDev vd = a.views[CHUNK ? sm.it.vidx : find_view(a.views, a.V, t)];
  if (CHUNK) {
    tx0 = sm.it.tx0;
    ty0 = sm.it.ty0;
  }
  if (STATS) {
    // block totals of list positions walked until the stop (the same count
    // with or without culling) and of blends (accumulator A)
    const uint2 rg = a.ranges[t];
    unsigned long long e = 0, bl2 = n_blend;
#pragma unroll
    for (int k = 0; k < PX; ++k)
      if ((inb >> k) & 1u) e += (A[k].done && walk_end[k] > 0) ? walk_end[k] : (rg.y - rg.x);
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
    int x, y, lvl;
    bool inside, in_band;
    float wband;
    pixel_of<B, FOV, PX>(a, vd, tx0, ty0, k, x, y, lvl, inside, in_band, wband);
    if (!inside) continue;
    const long long pix = vd.pix_base + (long long)y * vd.W + x;
    float r = fmaf(A[k].T, a.bg0, A[k].r), g = fmaf(A[k].T, a.bg1, A[k].g),
          bl = fmaf(A[k].T, a.bg2, A[k].b);
    if (FOV) {
      if (in_band) {
        const float rb = fmaf(Bq[k].T, a.bg0, Bq[k].r), gb = fmaf(Bq[k].T, a.bg1, Bq[k].g),
                    bb = fmaf(Bq[k].T, a.bg2, Bq[k].b);
        r = fmaf(wband, r - rb, rb);
        g = fmaf(wband, g - gb, gb);
        bl = fmaf(wband, bl - bb, bb);
      }
      a.T[2 * pix] = A[k].T;
      a.T[2 * pix + 1] = in_band ? Bq[k].T : 1.0f;
      a.last[2 * pix] = A[k].last;
      a.last[2 * pix + 1] = in_band ? Bq[k].last : -1;
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

// Whole tiles (CHUNK = false): one block per tile.  Chunked (CHUNK = true):
// persistent blocks take work items from a queue -- first the chunks of the
// heavy tiles, then the remaining tiles in order.
// Blocks per SM: foveated two-pixel blocks fill 768 threads (room for both
// accumulators' registers: no spills with 16 x 16 tiles, fewer with 8 x 8),
// the others 1024 (768 chunked).
template <int B, bool FOV, bool MV, bool STATS, int PX, bool CHUNK>
__global__ void __launch_bounds__(B * B / PX, ((FOV && PX == 2) || CHUNK ? 768 : 1024) /
                                                  (B * B / PX))
    k_render(RenderArgs a) {
  __shared__ RSmem<B, FOV, MV, STATS, PX> sm;
  const uint32_t *vals = *a.sel ? a.pval_b : a.pval_a;
  if (!CHUNK) {
    render_item<B, FOV, MV, STATS, PX, false>(a, sm, vals, blockIdx.x, 0, 0, 0);
    return;
  }
  const unsigned long long ns = min((unsigned long long)*a.n_slots, a.ch_cap);
  const unsigned long long total = ns + (unsigned long long)a.tiles;
  for (;;) {
    if (threadIdx.x == 0) sm.item = atomicAdd(a.queue, 1ull);
    __syncthreads();
    const unsigned long long item = sm.item;
    __syncthreads();
    if (item >= total) break;
    if (item < ns) {
      const uint2 cl = a.chunk_list[item];
      if (cl.y == kNoChunk) continue;   // slot of a tile that did not fit
      const uint2 rg = a.ranges[cl.x];
      const uint32_t nc = (rg.y - rg.x + (uint32_t)a.chunk - 1) / (uint32_t)a.chunk;
      render_item<B, FOV, MV, STATS, PX, true>(a, sm, vals, cl.x, cl.y, item, nc);
    } else {
      const long long t = (long long)(item - ns);
      if (a.chunk_tile[t].x != kNoChunk) continue;   // rendered as chunks
      render_item<B, FOV, MV, STATS, PX, true>(a, sm, vals, t, 0, 0, 0);
    }
  }
}

// Work list of the chunked render: a tile longer than `chunk` points gets
// ceil(len / chunk) consecutive chunk slots.  Tiles that do not fit the
// slot capacity are rendered whole (their slots are marked unused).
__global__ void k_chunk_plan(const uint2 *ranges, long long tiles, uint32_t chunk,
                             unsigned long long cap, uint32_t *n_slots, uint4 *chunk_tile,
                             uint2 *chunk_list) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < tiles;
       t += (long long)gridDim.x * blockDim.x) {
    const uint2 rg = ranges[t];
    const uint32_t len = rg.y - rg.x;
    uint32_t first = kNoChunk;
    if (len > chunk) {
      const uint32_t nc = (len + chunk - 1) / chunk;
      const unsigned long long b = atomicAdd(n_slots, nc);
      if (b + nc <= cap) {
        first = (uint32_t)b;
        for (uint32_t c = 0; c < nc; ++c) chunk_list[b + c] = make_uint2((uint32_t)t, c);
      } else {
        for (unsigned long long s = b; s < b + nc && s < cap; ++s)
          chunk_list[s] = make_uint2((uint32_t)t, kNoChunk);
      }
    }
    chunk_tile[t] = make_uint4(first, 0u, kNoChunk, 0u);
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
static void launch_t(const RenderArgs &a, long long tiles, bool chunked, int num_sms,
                     cudaStream_t s) {
  // two pixels per thread, except foveated renders with per-level parameters
  // or statistics, whose state does not fit the registers of two pixels
  constexpr int PX = (FOV && (MV || STATS)) ? 1 : 2;
  constexpr int NT = B * B / PX;
  if (STATS || !chunked) {
    k_render<B, FOV, MV, STATS, PX, false><<<(unsigned)tiles, NT, 0, s>>>(a);
    return;
  }
  // persistent blocks: as many as stay resident
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render<B, FOV, MV, false, PX, true>,
                                                      NT, 0) != cudaSuccess || per_sm < 1)
      per_sm = 1;
  }
  unsigned long long grid = (unsigned long long)per_sm * (unsigned long long)(num_sms > 0 ? num_sms : 1);
  const unsigned long long items = a.ch_cap + (unsigned long long)tiles;
  if (grid > items) grid = items;
  k_render<B, FOV, MV, false, PX, true><<<(unsigned)grid, NT, 0, s>>>(a);
}

template <int B>
static void launch_b(const RenderArgs &a, bool fov, bool mv, bool stats, long long tiles,
                     bool chunked, int num_sms, cudaStream_t s) {
  if (!fov) {
    if (stats) launch_t<B, false, false, true>(a, tiles, chunked, num_sms, s);
    else launch_t<B, false, false, false>(a, tiles, chunked, num_sms, s);
  } else if (!mv) {
    if (stats) launch_t<B, true, false, true>(a, tiles, chunked, num_sms, s);
    else launch_t<B, true, false, false>(a, tiles, chunked, num_sms, s);
  } else {
    if (stats) launch_t<B, true, true, true>(a, tiles, chunked, num_sms, s);
    else launch_t<B, true, true, false>(a, tiles, chunked, num_sms, s);
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
  a.mmfr = fov && (p->flags & GS_FLAG_MULTI_MODEL) ? 1 : 0;
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
  // heavy-tile chunking (not for statistics renders, whose per-point
  // counters need each tile walked once, in order)
  const bool chunked = p->chunk > 0 && !stats && p->bytes[R_CHUNK_PART] > 0;
  if (chunked) {
    a.chunk = p->chunk;
    a.tiles = p->tiles_total;
    a.chunk_list = region<uint2>(p, ws, R_WORK);
    a.chunk_tile = region<uint4>(p, ws, R_CHUNK_TILE);
    a.part_ct = region<float4>(p, ws, R_CHUNK_PART);
    a.part_last = region<int32_t>(p, ws, R_CHUNK_LAST);
    a.ch_cap = (unsigned long long)p->chunk_cap;
    a.n_slots = &hdr->n_slots;
    a.queue = &hdr->queue;
    cudaError_t e = cudaMemsetAsync(&hdr->queue, 0, sizeof(unsigned long long) + sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const long long T = p->tiles_total;
    const unsigned blocks = (unsigned)((T + 255) / 256 < 4096 ? (T + 255) / 256 : 4096);
    k_chunk_plan<<<blocks, 256, 0, s>>>(a.ranges, T, (uint32_t)p->chunk, a.ch_cap, &hdr->n_slots,
                                        a.chunk_tile, region<uint2>(p, ws, R_WORK));
  }
  if (p->tile == 16)
    launch_b<16>(a, fov, mv, stats != nullptr, p->tiles_total, chunked, p->num_sms, s);
  else
    launch_b<8>(a, fov, mv, stats != nullptr, p->tiles_total, chunked, p->num_sms, s);
  return cudaGetLastError();
}

}  // namespace gs
