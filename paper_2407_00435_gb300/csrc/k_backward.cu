// k_backward.cu -- adjoint of the rasterizer, for retraining through the
// renderer (the pruning and foveated levels of Sec. 3.4 and Sec. 4.3 are
// obtained by training through it).
//
// Pass 1 (k_render_bwd_plain for plain views: two pixels per thread and
// per-warp lists of the points that reach the warp; k_render_bwd for
// foveated views: one pixel per thread, two accumulators): one block per
// tile, walking the tile's list back to front from the last blended point.
// With the forward's final transmittance T_N and the colour S accumulated
// behind a point (starting at T_N bg), each blended point i gives
//   dL/dc_i     = T_i alpha_i g
//   dL/dalpha_i = g . (T_i c_i - S / (1 - alpha_i)),   T_i = T_{i+1} / (1 - alpha_i)
// and, below the 0.99 clamp, dL/dopacity = dL/dalpha alpha / o and
// dL/dpower = dL/dalpha alpha with power = -1/2 d^T Q d, d = p - mu:
//   dL/dmu = dL/dpower Q d,   dL/dQ = -1/2 dL/dpower d d^T.
// Contributions are summed over each warp by a reduce-scatter of shuffles,
// then over the block in shared memory, then added once per (tile, point)
// to a per-item gradient record.
//
// Pass 2 (k_project_bwd): one thread per visible item chains the 2D
// gradients to the 3D parameters (mean, scale, rotation, opacity, SH) through
// Sigma' = G G^T + 0.3 I, G = J W Rq diag(s), and the SH view direction.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_internal.cuh"
#include "raster.cuh"

namespace gs {

constexpr float kY00b = 0.28209479177387814f;
constexpr int kGradItem = 12;   // floats per item: dmu(2) dQ(3) do(1) dc(3) pad(3)
constexpr int kGradLv = 4;      // floats per (level, item): do(1) dc(3)

struct BwdArgs {
  const ViewDev *views;
  int V;
  long long n;
  const uint2 *ranges;
  const uint32_t *pval_a, *pval_b;
  const uint32_t *sel;
  const float4 *rec_mean, *rec_shape, *rec_color, *rec_rest;
  const uint32_t *rec_gid;
  const uint8_t *rec_m;
  const float *opac;          // base opacities (N)
  int L;
  float band;
  int mmfr;                   // a separate model per level (GS_FLAG_MULTI_MODEL)
  const float *opacity_lv, *dc_lv;
  float bg0, bg1, bg2;
  const float *dL;            // (P,3)
  const float *T;             // (P) or (P,2)
  const int32_t *last;        // (P) or (P,2)
  float *grad_item;           // (M, kGradItem)
  float *grad_lv;             // (L-1, M, kGradLv) or null
  long long max_visible;
};

struct BAcc {
  float T, Sr, Sg, Sb;   // transmittance after the current point; colour behind it
  float gr, gg, gb;      // upstream gradient of this accumulator's colour
  int last;
};

// Sums of nine per-lane values over the warp by reduce-scatter: each
// halving step keeps half of the values and adds the partner's copy of them
// (16 shuffles in all); lanes 2i and 2i + 1 end with the total of value i,
// which is returned (value index lane >> 1; lanes >= 18 return 0).
__device__ __forceinline__ float warp_reduce_scatter9(const float (&v)[9], int lane) {
  float r[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) r[k] = k < 9 ? v[k] : 0.0f;
#pragma unroll
  for (int off = 16, h = 8; off >= 2; off >>= 1, h >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? r[i] : r[i + h];
      const float keep = up ? r[i + h] : r[i];
      r[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return r[0] + __shfl_xor_sync(0xffffffffu, r[0], 1);
}

template <int B, bool FOV, bool MV>
__global__ void __launch_bounds__(B * B) k_render_bwd(BwdArgs a) {
  constexpr int NT = B * B;
  __shared__ float2 s_mean[NT];
  __shared__ float4 s_shape[NT];
  __shared__ float4 s_col[NT];
  __shared__ float s_op[NT];
  __shared__ uint32_t s_j[NT];
  __shared__ int s_m[FOV ? NT : 1];
  __shared__ float4 s_lv[MV ? NT : 1][MV ? kMvMaxLevels - 1 : 1];
  __shared__ float s_g[NT][9];   // per batch slot: dmu(2) dQ(3) do(1) dc(3)
  __shared__ float4 s_ea[NT], s_eb[NT];   // evaluation records (as in the forward)
  __shared__ int s_maxlast;

  const long long t = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const ViewDev vd = a.views[find_view(a.views, a.V, t)];
  const int local = (int)(t - vd.tile_base);
  const int tx0 = (local % vd.tx) * B, ty0 = (local / vd.tx) * B;
  const int lx = (warp % WarpGeom<B, 1>::kWx) * 8 + (lane & 7);
  const int ly = (warp / WarpGeom<B, 1>::kWx) * 4 + (lane >> 3);
  const int x = tx0 + lx, y = ty0 + ly;
  const bool inside = x < vd.W && y < vd.H;
  const float px = (float)lx + 0.5f, py = (float)ly + 0.5f;
  int lvl = 1;
  bool in_band = false;
  float wband = 1.0f;
  if (FOV) pixel_level(vd, a.L, a.band, x, y, lvl, in_band, wband);

  BAcc A = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -1};
  BAcc Bq = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -1};
  if (inside) {
    const long long pix = vd.pix_base + (long long)y * vd.W + x;
    const float g0 = a.dL[3 * pix], g1 = a.dL[3 * pix + 1], g2 = a.dL[3 * pix + 2];
    const float wa = FOV && in_band ? wband : 1.0f;
    if (FOV) {
      A.T = a.T[2 * pix];
      A.last = a.last[2 * pix];
      if (in_band) {
        Bq.T = a.T[2 * pix + 1];
        Bq.last = a.last[2 * pix + 1];
      }
    } else {
      A.T = a.T[pix];
      A.last = a.last[pix];
    }
    A.gr = wa * g0; A.gg = wa * g1; A.gb = wa * g2;
    A.Sr = A.T * a.bg0; A.Sg = A.T * a.bg1; A.Sb = A.T * a.bg2;
    if (FOV && in_band) {
      const float wb = 1.0f - wband;
      Bq.gr = wb * g0; Bq.gg = wb * g1; Bq.gb = wb * g2;
      Bq.Sr = Bq.T * a.bg0; Bq.Sg = Bq.T * a.bg1; Bq.Sb = Bq.T * a.bg2;
    }
  }
  if (tid == 0) s_maxlast = -1;
  __syncthreads();
  atomicMax(&s_maxlast, max(A.last, Bq.last));
  for (int k = tid; k < NT * 9; k += NT) (&s_g[0][0])[k] = 0.0f;
  __syncthreads();
  const uint2 rg = a.ranges[t];
  const uint32_t *vals = *a.sel ? a.pval_b : a.pval_a;
  const int maxlast = s_maxlast;
  if (maxlast < 0) return;
  const uint32_t end = rg.x + (uint32_t)maxlast + 1;

  for (uint32_t hi = end; hi > rg.x;) {
    const uint32_t lo = hi - rg.x > (uint32_t)NT ? hi - NT : rg.x;
    const uint32_t cnt = hi - lo;
    if ((uint32_t)tid < cnt) {
      const uint32_t j = vals[lo + tid];
      const float4 mean = a.rec_mean[j];
      s_mean[tid] = make_float2((mean.x - (float)tx0) + mean.z, (mean.y - (float)ty0) + mean.w);
      s_shape[tid] = a.rec_shape[j];
      const float4 col = a.rec_color[j];
      s_col[tid] = col;
      s_j[tid] = j;
      const uint32_t gid = a.rec_gid[j];
      s_op[tid] = a.opac[gid];
      if (FOV) s_m[tid] = a.rec_m[j];
      float Fmax = col.w;
      if (MV) {
        const float4 rest = a.rec_rest[j];
        for (int l = 2; l <= a.L; ++l) {
          float o = a.opac[gid];
          float4 c = col;
          if (a.opacity_lv) o = a.opacity_lv[(long long)(l - 2) * a.n + gid];
          if (a.dc_lv) {
            const float *dc = a.dc_lv + ((long long)(l - 2) * a.n + gid) * 3;
            c.x = fmaxf(0.0f, fmaf(kY00b, dc[0], rest.x) + kShOffset);
            c.y = fmaxf(0.0f, fmaf(kY00b, dc[1], rest.y) + kShOffset);
            c.z = fmaxf(0.0f, fmaf(kY00b, dc[2], rest.z) + kShOffset);
          }
          // .w keeps log2 o as in the forward
          s_lv[tid][l - 2] = make_float4(c.x, c.y, c.z, a.opacity_lv ? log2f(o) : col.w);
          Fmax = fmaxf(Fmax, s_lv[tid][l - 2].w);
        }
      }
      float4 ea, eb;
      make_eval(s_mean[tid].x, s_mean[tid].y, s_shape[tid], col.w,
                warp_mask<B, 1>(s_mean[tid].x, s_mean[tid].y, s_shape[tid], Fmax), ea, eb);
      s_ea[tid] = ea;
      s_eb[tid] = eb;
    }
    __syncthreads();
    for (int q = (int)cnt - 1; q >= 0; --q) {
      const float4 eb = s_eb[q];
      if (!((__float_as_uint(eb.w) >> warp) & 1u)) continue;   // cannot reach this warp's pixels
      const int pos = (int)(lo - rg.x) + q;
      const float2 mu = s_mean[q];
      const float4 sh = s_shape[q];
      float t1, t2;
      const float sq = eval_s(px, py, s_ea[q], eb, t1, t2);
      const float dx = px - mu.x, dy = py - mu.y;
      const int m = FOV ? s_m[q] : 0;
      float gmx = 0.f, gmy = 0.f, gqa = 0.f, gqb = 0.f, gqc = 0.f, gop = 0.f, gcr = 0.f,
            gcg = 0.f, gcb = 0.f;
#pragma unroll
      for (int acc = 0; acc < (FOV ? 2 : 1); ++acc) {
        BAcc &S = acc == 0 ? A : Bq;
        const int L_here = acc == 0 ? lvl : lvl - 1;
        if (pos > S.last) continue;
        if (FOV && !takes_part(m, L_here, a.mmfr)) continue;
        const bool own = MV && L_here >= 2;
        const float4 c = own ? s_lv[q][L_here - 2] : s_col[q];
        const float r2 = own ? __fsub_rn(c.w, kLog2AlphaMin) : eb.z;
        if (!(sq <= r2)) continue;
        const float al = alpha_of(__fsub_rn(c.w, sq));
        const float rom = 1.0f / (1.0f - al);
        const float Tb = S.T * rom;
        const float w = al * Tb;
        const float dcr = w * S.gr, dcg = w * S.gg, dcb = w * S.gb;
        const float dal = S.gr * (Tb * c.x - S.Sr * rom) + S.gg * (Tb * c.y - S.Sg * rom) +
                          S.gb * (Tb * c.z - S.Sb * rom);
        S.Sr = fmaf(w, c.x, S.Sr);
        S.Sg = fmaf(w, c.y, S.Sg);
        S.Sb = fmaf(w, c.z, S.Sb);
        S.T = Tb;
        float dop = 0.0f;
        if (al < kAlphaMax) {
          const float o = (own && a.opacity_lv) ? exp2f(c.w) : s_op[q];
          dop = dal * al / o;
          const float dpow = dal * al;
          // Q d = (w1 t1 + w2 t2) / kWhiten^2, d = pixel - mean
          const float inv = 1.0f / (kWhiten * kWhiten);
          gmx += dpow * (sh.x * t1 + sh.z * t2) * inv;
          gmy += dpow * (sh.y * t1 + sh.w * t2) * inv;
          gqa += -0.5f * dpow * dx * dx;
          gqb += -dpow * dx * dy;
          gqc += -0.5f * dpow * dy * dy;
        }
        if (own) {
          // this level's own opacity / DC (multi-versioned): added per pixel
          float *g = a.grad_lv + ((long long)(L_here - 2) * a.max_visible + s_j[q]) * kGradLv;
          if (dop != 0.f) atomicAdd(&g[0], dop);
          atomicAdd(&g[1], dcr);
          atomicAdd(&g[2], dcg);
          atomicAdd(&g[3], dcb);
        } else {
          gop += dop; gcr += dcr; gcg += dcg; gcb += dcb;
        }
      }
      const bool any = __any_sync(0xffffffffu, gmx != 0.f || gmy != 0.f || gqa != 0.f ||
                                                    gqb != 0.f || gqc != 0.f || gop != 0.f ||
                                                    gcr != 0.f || gcg != 0.f || gcb != 0.f);
      if (any) {
        const float v[9] = {gmx, gmy, gqa, gqb, gqc, gop, gcr, gcg, gcb};
        const float tot = warp_reduce_scatter9(v, lane);
        const int idx = lane >> 1;
        if ((lane & 1) == 0 && idx < 9 && tot != 0.f) atomicAdd(&s_g[q][idx], tot);
      }
    }
    __syncthreads();
    // flush this batch's per-point sums (one add per value per tile)
    if ((uint32_t)tid < cnt) {
      float *g = a.grad_item + (long long)s_j[tid] * kGradItem;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float v = s_g[tid][k];
        if (v != 0.f) atomicAdd(&g[k], v);
        s_g[tid][k] = 0.f;
      }
    }
    __syncthreads();
    hi = lo;
  }
}

// Plain views: the forward's layout (two pixels per thread, rows 4 apart),
// per-warp ordered lists of the batch points that can reach the warp's
// pixels and lie at or before the last position any of them blended, and a
// reduce-scatter of the nine per-point sums over the warp (16 shuffles; the
// two lanes holding a total, the even one adds it to shared memory).
template <int B>
struct BwdSmem {
  static constexpr int PX = 2;
  static constexpr int NT = B * B / PX;                   // threads
  static constexpr int NB = 2 * NT < 256 ? 2 * NT : 256;  // points per batch
  static constexpr int SPT = NB / NT;                     // staged per thread
  static constexpr int NWS = NT / 32;                     // staging warps
  static constexpr int NW = WarpGeom<B, PX>::kWarps;      // pixel warps
  float2 mean[NB];
  float4 shape[NB];
  float4 col[NB];
  float4 ea[NB], eb[NB];
  float op[NB];
  uint32_t j[NB];
  float g[NB][9];   // per batch slot: dmu(2) dQ(3) do(1) dc(3)
  uint16_t list[NW][NB];
  uint16_t wcnt[NW][SPT * NWS];
  uint16_t woff[NW][SPT * NWS + 1];
  int wlast[NW];    // last blended position of the warp's pixels (-1: none)
  int maxlast;
};

template <int B>
__global__ void __launch_bounds__(B * B / 2) k_render_bwd_plain(BwdArgs a) {
  using Sm = BwdSmem<B>;
  using G = WarpGeom<B, 2>;
  constexpr int NT = Sm::NT, NB = Sm::NB, SPT = Sm::SPT, NWS = Sm::NWS, NW = Sm::NW;
  __shared__ Sm sm;
  const long long t = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t ltmask = (1u << lane) - 1u;
  const ViewDev vd = a.views[find_view(a.views, a.V, t)];
  const int local = (int)(t - vd.tile_base);
  const int tx0 = (local % vd.tx) * B, ty0 = (local / vd.tx) * B;
  const int lx = (warp % G::kWx) * 8 + (lane & 7);
  const int ly0 = (warp / G::kWx) * G::kRows + (lane >> 3);
  const float px = (float)lx + 0.5f;
  float py[2];
  BAcc A[2];
  int mylast = -1;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int x = tx0 + lx, y = ty0 + ly0 + 4 * k;
    py[k] = (float)(ly0 + 4 * k) + 0.5f;
    A[k] = BAcc{1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -1};
    if (x < vd.W && y < vd.H) {
      const long long pix = vd.pix_base + (long long)y * vd.W + x;
      A[k].T = a.T[pix];
      A[k].last = a.last[pix];
      A[k].gr = a.dL[3 * pix];
      A[k].gg = a.dL[3 * pix + 1];
      A[k].gb = a.dL[3 * pix + 2];
      A[k].Sr = A[k].T * a.bg0;
      A[k].Sg = A[k].T * a.bg1;
      A[k].Sb = A[k].T * a.bg2;
      mylast = max(mylast, A[k].last);
    }
  }
  int wl = mylast;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
  if (tid == 0) sm.maxlast = -1;
  for (int k = tid; k < NB * 9; k += NT) (&sm.g[0][0])[k] = 0.0f;
  __syncthreads();
  if (lane == 0) {
    sm.wlast[warp] = wl;
    atomicMax(&sm.maxlast, wl);
  }
  __syncthreads();
  const int maxlast = sm.maxlast;
  if (maxlast < 0) return;
  const uint2 rg = a.ranges[t];
  const uint32_t *vals = *a.sel ? a.pval_b : a.pval_a;
  const uint32_t end = rg.x + (uint32_t)maxlast + 1;
  const float inv = 1.0f / (kWhiten * kWhiten);

  for (uint32_t hi = end; hi > rg.x;) {
    const uint32_t lo = hi - rg.x > (uint32_t)NB ? hi - NB : rg.x;
    const uint32_t cnt = hi - lo;
    const int base = (int)(lo - rg.x);
    // stage the batch: records, evaluation constants and the warps each
    // point can reach at or before their last blended position
    uint32_t wm[SPT];
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int q = tid + u * NT;
      wm[u] = 0u;
      if ((uint32_t)q < cnt) {
        const uint32_t j = vals[lo + q];
        const float4 mean = a.rec_mean[j];
        const float mx = (mean.x - (float)tx0) + mean.z, my = (mean.y - (float)ty0) + mean.w;
        const float4 shp = a.rec_shape[j];
        const float4 col = a.rec_color[j];
        sm.mean[q] = make_float2(mx, my);
        sm.shape[q] = shp;
        sm.col[q] = col;
        sm.j[q] = j;
        sm.op[q] = 1.0f / a.opac[a.rec_gid[j]];   // reciprocal opacity
        uint32_t msk = warp_mask_exact<B, 2>(mx, my, shp, col.w);
#pragma unroll
        for (int w = 0; w < NW; ++w)
          if (base + q > sm.wlast[w]) msk &= ~(1u << w);
        float4 ea, eb;
        make_eval(mx, my, shp, col.w, msk, ea, eb);
        sm.ea[q] = ea;
        sm.eb[q] = eb;
        wm[u] = msk;
      }
    }
    // ordered per-warp lists (ballot prefixes, then prefix sums over the
    // (slot group, staging warp) pairs)
    uint32_t pfx[SPT][NW];
#pragma unroll
    for (int u = 0; u < SPT; ++u)
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t bal = __ballot_sync(0xffffffffu, (wm[u] >> w) & 1u);
        pfx[u][w] = __popc(bal & ltmask);
        if (lane == 0) sm.wcnt[w][u * NWS + warp] = (uint16_t)__popc(bal);
      }
    __syncthreads();
    if (tid < NW) {
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
      for (int w = 0; w < NW; ++w)
        if ((wm[u] >> w) & 1u)
          sm.list[w][sm.woff[w][u * NWS + warp] + pfx[u][w]] = (uint16_t)(tid + u * NT);
    __syncthreads();
    // back to front over this warp's list
    const int nlist = sm.woff[warp][SPT * NWS];
    for (int li = nlist - 1; li >= 0; --li) {
      const int q = sm.list[warp][li];
      const int pos = base + q;
      const float4 ea = sm.ea[q], eb = sm.eb[q], c = sm.col[q], shp = sm.shape[q];
      const float2 mu = sm.mean[q];
      const float io = sm.op[q];
      float v[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) v[k] = 0.0f;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        BAcc &S = A[k];
        if (pos > S.last) continue;
        float t1, t2;
        const float sq = eval_s(px, py[k], ea, eb, t1, t2);
        if (!(sq <= eb.z)) continue;
        const float al = alpha_of(__fsub_rn(c.w, sq));
        const float rom = 1.0f / (1.0f - al);
        const float Tb = S.T * rom;
        const float w = al * Tb;
        v[6] += w * S.gr;
        v[7] += w * S.gg;
        v[8] += w * S.gb;
        const float dal = S.gr * (Tb * c.x - S.Sr * rom) + S.gg * (Tb * c.y - S.Sg * rom) +
                          S.gb * (Tb * c.z - S.Sb * rom);
        S.Sr = fmaf(w, c.x, S.Sr);
        S.Sg = fmaf(w, c.y, S.Sg);
        S.Sb = fmaf(w, c.z, S.Sb);
        S.T = Tb;
        if (al < kAlphaMax) {
          const float dpow = dal * al;
          const float dx = px - mu.x, dy = py[k] - mu.y;
          v[5] += dpow * io;
          // Q d = (w1 t1 + w2 t2) / kWhiten^2, d = pixel - mean
          v[0] += dpow * (shp.x * t1 + shp.z * t2) * inv;
          v[1] += dpow * (shp.y * t1 + shp.w * t2) * inv;
          v[2] += -0.5f * dpow * dx * dx;
          v[3] += -dpow * dx * dy;
          v[4] += -0.5f * dpow * dy * dy;
        }
      }
      bool nz = false;
#pragma unroll
      for (int k = 0; k < 9; ++k) nz = nz || v[k] != 0.0f;
      if (__any_sync(0xffffffffu, nz)) {
        const float tot = warp_reduce_scatter9(v, lane);
        const int idx = lane >> 1;
        if ((lane & 1) == 0 && idx < 9 && tot != 0.0f) atomicAdd(&sm.g[q][idx], tot);
      }
    }
    __syncthreads();
    // flush this batch's per-point sums (one add per value per tile)
    for (int q = tid; q < (int)cnt; q += NT) {
      float *g = a.grad_item + (long long)sm.j[q] * kGradItem;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float v = sm.g[q][k];
        if (v != 0.f) atomicAdd(&g[k], v);
        sm.g[q][k] = 0.f;
      }
    }
    __syncthreads();
    hi = lo;
  }
}

// One blend of the back-to-front replay of accumulator S (alpha al, 1 / (1 -
// al) = rom, colour c): adds dL/dc to v[6..8], updates S and returns dL/dalpha.
__device__ __forceinline__ float bwd_blend(BAcc &S, float al, float rom, float4 c, float (&v)[9]) {
  const float Tb = S.T * rom;
  const float w = al * Tb;
  v[6] += w * S.gr;
  v[7] += w * S.gg;
  v[8] += w * S.gb;
  const float dal = S.gr * (Tb * c.x - S.Sr * rom) + S.gg * (Tb * c.y - S.Sg * rom) +
                    S.gb * (Tb * c.z - S.Sb * rom);
  S.Sr = fmaf(w, c.x, S.Sr);
  S.Sg = fmaf(w, c.y, S.Sg);
  S.Sb = fmaf(w, c.z, S.Sb);
  S.T = Tb;
  return dal;
}

// Foveated views without per-level parameters, in the plain kernel's layout
// (two pixels per thread, per-warp ordered lists): each pixel replays its own
// level's accumulator and, inside a blend band, the level below's (both in
// registers).  A point enters a warp's list only if it can reach the warp's
// pixels, lies at or before the last position they blended, and takes part
// in a level one of them composites.
template <int B>
__global__ void __launch_bounds__(B * B / 2) k_render_bwd_fov(BwdArgs a) {
  using Sm = BwdSmem<B>;
  using G = WarpGeom<B, 2>;
  constexpr int NT = Sm::NT, NB = Sm::NB, SPT = Sm::SPT, NWS = Sm::NWS, NW = Sm::NW;
  __shared__ Sm sm;
  __shared__ uint32_t s_wlv[NW];   // levels the warp's pixels composite (bit l)
  __shared__ uint8_t s_m[NB];
  const long long t = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t ltmask = (1u << lane) - 1u;
  const ViewDev vd = a.views[find_view(a.views, a.V, t)];
  const int local = (int)(t - vd.tile_base);
  const int tx0 = (local % vd.tx) * B, ty0 = (local / vd.tx) * B;
  const int lx = (warp % G::kWx) * 8 + (lane & 7);
  const int ly0 = (warp / G::kWx) * G::kRows + (lane >> 3);
  const float px = (float)lx + 0.5f;
  const bool mmfr = a.mmfr != 0;
  float py[2];
  int lvl[2];
  bool band[2];
  BAcc A[2], Bq[2];
  int mylast = -1;
  uint32_t mylv = 0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int x = tx0 + lx, y = ty0 + ly0 + 4 * k;
    py[k] = (float)(ly0 + 4 * k) + 0.5f;
    A[k] = BAcc{1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -1};
    Bq[k] = A[k];
    lvl[k] = 1;
    band[k] = false;
    if (x < vd.W && y < vd.H) {
      float wband = 1.0f;
      pixel_level(vd, a.L, a.band, x, y, lvl[k], band[k], wband);
      const long long pix = vd.pix_base + (long long)y * vd.W + x;
      const float g0 = a.dL[3 * pix], g1 = a.dL[3 * pix + 1], g2 = a.dL[3 * pix + 2];
      const float wa = band[k] ? wband : 1.0f;
      A[k].T = a.T[2 * pix];
      A[k].last = a.last[2 * pix];
      A[k].gr = wa * g0; A[k].gg = wa * g1; A[k].gb = wa * g2;
      A[k].Sr = A[k].T * a.bg0; A[k].Sg = A[k].T * a.bg1; A[k].Sb = A[k].T * a.bg2;
      mylast = max(mylast, A[k].last);
      mylv |= 1u << lvl[k];
      if (band[k]) {
        const float wb = 1.0f - wband;
        Bq[k].T = a.T[2 * pix + 1];
        Bq[k].last = a.last[2 * pix + 1];
        Bq[k].gr = wb * g0; Bq[k].gg = wb * g1; Bq[k].gb = wb * g2;
        Bq[k].Sr = Bq[k].T * a.bg0; Bq[k].Sg = Bq[k].T * a.bg1; Bq[k].Sb = Bq[k].T * a.bg2;
        mylast = max(mylast, Bq[k].last);
        mylv |= 1u << (lvl[k] - 1);
      }
    }
  }
  int wl = mylast;
  uint32_t wlv = mylv;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
    wlv |= __shfl_xor_sync(0xffffffffu, wlv, o);
  }
  if (tid == 0) sm.maxlast = -1;
  for (int k = tid; k < NB * 9; k += NT) (&sm.g[0][0])[k] = 0.0f;
  __syncthreads();
  if (lane == 0) {
    sm.wlast[warp] = wl;
    s_wlv[warp] = wlv;
    atomicMax(&sm.maxlast, wl);
  }
  __syncthreads();
  const int maxlast = sm.maxlast;
  if (maxlast < 0) return;
  const uint2 rg = a.ranges[t];
  const uint32_t *vals = *a.sel ? a.pval_b : a.pval_a;
  const uint32_t end = rg.x + (uint32_t)maxlast + 1;
  const float inv = 1.0f / (kWhiten * kWhiten);

  for (uint32_t hi = end; hi > rg.x;) {
    const uint32_t lo = hi - rg.x > (uint32_t)NB ? hi - NB : rg.x;
    const uint32_t cnt = hi - lo;
    const int base = (int)(lo - rg.x);
    uint32_t wm[SPT];
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int q = tid + u * NT;
      wm[u] = 0u;
      if ((uint32_t)q < cnt) {
        const uint32_t j = vals[lo + q];
        const float4 mean = a.rec_mean[j];
        const float mx = (mean.x - (float)tx0) + mean.z, my = (mean.y - (float)ty0) + mean.w;
        const float4 shp = a.rec_shape[j];
        const float4 col = a.rec_color[j];
        const int m = a.rec_m[j];
        sm.mean[q] = make_float2(mx, my);
        sm.shape[q] = shp;
        sm.col[q] = col;
        sm.j[q] = j;
        s_m[q] = (uint8_t)m;
        sm.op[q] = 1.0f / a.opac[a.rec_gid[j]];   // reciprocal opacity
        // levels the point takes part in (bit l)
        const uint32_t pm = mmfr ? (1u << m) : ((2u << m) - 2u);
        uint32_t msk = warp_mask_exact<B, 2>(mx, my, shp, col.w);
#pragma unroll
        for (int w = 0; w < NW; ++w)
          if (base + q > sm.wlast[w] || !(pm & s_wlv[w])) msk &= ~(1u << w);
        float4 ea, eb;
        make_eval(mx, my, shp, col.w, msk, ea, eb);
        sm.ea[q] = ea;
        sm.eb[q] = eb;
        wm[u] = msk;
      }
    }
    uint32_t pfx[SPT][NW];
#pragma unroll
    for (int u = 0; u < SPT; ++u)
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t bal = __ballot_sync(0xffffffffu, (wm[u] >> w) & 1u);
        pfx[u][w] = __popc(bal & ltmask);
        if (lane == 0) sm.wcnt[w][u * NWS + warp] = (uint16_t)__popc(bal);
      }
    __syncthreads();
    if (tid < NW) {
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
      for (int w = 0; w < NW; ++w)
        if ((wm[u] >> w) & 1u)
          sm.list[w][sm.woff[w][u * NWS + warp] + pfx[u][w]] = (uint16_t)(tid + u * NT);
    __syncthreads();
    const int nlist = sm.woff[warp][SPT * NWS];
    for (int li = nlist - 1; li >= 0; --li) {
      const int q = sm.list[warp][li];
      const int pos = base + q;
      const float4 ea = sm.ea[q], eb = sm.eb[q], c = sm.col[q], shp = sm.shape[q];
      const float2 mu = sm.mean[q];
      const float io = sm.op[q];
      const int m = s_m[q];
      float v[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) v[k] = 0.0f;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const bool useA = pos <= A[k].last && takes_part(m, lvl[k], mmfr);
        const bool useB = band[k] && pos <= Bq[k].last && takes_part(m, lvl[k] - 1, mmfr);
        if (!useA && !useB) continue;
        float t1, t2;
        const float sq = eval_s(px, py[k], ea, eb, t1, t2);
        if (!(sq <= eb.z)) continue;
        const float al = alpha_of(__fsub_rn(c.w, sq));
        const float rom = 1.0f / (1.0f - al);
        float dal = 0.0f;
        if (useA) dal += bwd_blend(A[k], al, rom, c, v);
        if (useB) dal += bwd_blend(Bq[k], al, rom, c, v);
        if (al < kAlphaMax) {
          const float dpow = dal * al;
          const float dx = px - mu.x, dy = py[k] - mu.y;
          v[5] += dpow * io;
          v[0] += dpow * (shp.x * t1 + shp.z * t2) * inv;
          v[1] += dpow * (shp.y * t1 + shp.w * t2) * inv;
          v[2] += -0.5f * dpow * dx * dx;
          v[3] += -dpow * dx * dy;
          v[4] += -0.5f * dpow * dy * dy;
        }
      }
      bool nz = false;
#pragma unroll
      for (int k = 0; k < 9; ++k) nz = nz || v[k] != 0.0f;
      if (__any_sync(0xffffffffu, nz)) {
        const float tot = warp_reduce_scatter9(v, lane);
        const int idx = lane >> 1;
        if ((lane & 1) == 0 && idx < 9 && tot != 0.0f) atomicAdd(&sm.g[q][idx], tot);
      }
    }
    __syncthreads();
    for (int q = tid; q < (int)cnt; q += NT) {
      float *g = a.grad_item + (long long)sm.j[q] * kGradItem;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float v = sm.g[q][k];
        if (v != 0.f) atomicAdd(&g[k], v);
        sm.g[q][k] = 0.f;
      }
    }
    __syncthreads();
    hi = lo;
  }
}

// ---------------------------------------------------------------------------
// pass 2: chain to 3D parameters
// ---------------------------------------------------------------------------
struct PBwdArgs {
  long long n;
  int S;
  const float *means, *scales, *quats, *opac, *sh;
  const gs_camera *cams;
  const ViewDev *views;
  const unsigned long long *n_items;
  long long max_visible;
  const uint32_t *rec_gid, *rec_view, *rec_depth;
  const float4 *rec_shape;
  const float *grad_item, *grad_lv;
  int L;
  const float *opacity_lv, *dc_lv;
  float *d_means, *d_scales, *d_quats, *d_opac, *d_sh, *d_opac_lv, *d_dc_lv;
};

// gradient of the SH basis polynomials (degree <= 3) with respect to the
// direction components, treated as independent
__device__ __forceinline__ void sh_basis_and_grad(float x, float y, float z, int S, float Y[16],
                                                  float dY[16][3]) {
  const float k1 = 0.48860251190291992f, k2a = 1.0925484305920792f, k2b = 0.31539156525252005f,
              k2c = 0.54627421529603959f, k3a = 0.59004358992664352f, k3b = 2.8906114426405538f,
              k3c = 0.45704579946446572f, k3d = 0.37317633259011546f, k3e = 1.4453057213202769f;
#pragma unroll
  for (int k = 0; k < 16; ++k) { Y[k] = 0.f; dY[k][0] = dY[k][1] = dY[k][2] = 0.f; }
  Y[0] = kY00b;
  if (S > 1) {
    Y[1] = -k1 * y; dY[1][1] = -k1;
    Y[2] = k1 * z; dY[2][2] = k1;
    Y[3] = -k1 * x; dY[3][0] = -k1;
  }
  const float xx = x * x, yy = y * y, zz = z * z;
  if (S > 4) {
    Y[4] = k2a * x * y; dY[4][0] = k2a * y; dY[4][1] = k2a * x;
    Y[5] = -k2a * y * z; dY[5][1] = -k2a * z; dY[5][2] = -k2a * y;
    Y[6] = k2b * (2.f * zz - xx - yy);
    dY[6][0] = -2.f * k2b * x; dY[6][1] = -2.f * k2b * y; dY[6][2] = 4.f * k2b * z;
    Y[7] = -k2a * x * z; dY[7][0] = -k2a * z; dY[7][2] = -k2a * x;
    Y[8] = k2c * (xx - yy); dY[8][0] = 2.f * k2c * x; dY[8][1] = -2.f * k2c * y;
  }
  if (S > 9) {
    Y[9] = -k3a * y * (3.f * xx - yy);
    dY[9][0] = -6.f * k3a * x * y; dY[9][1] = -k3a * (3.f * xx - 3.f * yy);
    Y[10] = k3b * x * y * z;
    dY[10][0] = k3b * y * z; dY[10][1] = k3b * x * z; dY[10][2] = k3b * x * y;
    Y[11] = -k3c * y * (4.f * zz - xx - yy);
    dY[11][0] = 2.f * k3c * x * y; dY[11][1] = -k3c * (4.f * zz - xx - 3.f * yy);
    dY[11][2] = -8.f * k3c * y * z;
    Y[12] = k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    dY[12][0] = -6.f * k3d * x * z; dY[12][1] = -6.f * k3d * y * z;
    dY[12][2] = k3d * (6.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -k3c * x * (4.f * zz - xx - yy);
    dY[13][0] = -k3c * (4.f * zz - 3.f * xx - yy); dY[13][1] = 2.f * k3c * x * y;
    dY[13][2] = -8.f * k3c * x * z;
    Y[14] = k3e * z * (xx - yy);
    dY[14][0] = 2.f * k3e * x * z; dY[14][1] = -2.f * k3e * y * z; dY[14][2] = k3e * (xx - yy);
    Y[15] = -k3a * x * (xx - 3.f * yy);
    dY[15][0] = -k3a * (3.f * xx - 3.f * yy); dY[15][1] = 6.f * k3a * x * y;
  }
}

template <int S>
__global__ void __launch_bounds__(128) k_project_bwd(PBwdArgs a) {
  const unsigned long long nn = *a.n_items;
  const long long M = (long long)nn > a.max_visible ? a.max_visible : (long long)nn;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < M;
       j += (long long)gridDim.x * blockDim.x) {
    if (a.rec_depth[j] == 0xffffffffu) continue;   // invisible slot
    const float *gi = a.grad_item + j * kGradItem;
    const float gmx = gi[0], gmy = gi[1], gqa = gi[2], gqb = gi[3], gqc = gi[4], gop = gi[5];
    const float gc[3] = {gi[6], gi[7], gi[8]};
    const long long i = a.rec_gid[j];
    const int v = (int)a.rec_view[j];
    const gs_camera cam = a.cams[v];
    const ViewDev &vd = a.views[v];
    const float mu[3] = {a.means[3 * i], a.means[3 * i + 1], a.means[3 * i + 2]};
    const float s[3] = {a.scales[3 * i], a.scales[3 * i + 1], a.scales[3 * i + 2]};
    float qv[4] = {a.quats[4 * i], a.quats[4 * i + 1], a.quats[4 * i + 2], a.quats[4 * i + 3]};
    const float *R = cam.R;
    // camera-space mean
    const float pcx = R[0] * mu[0] + R[1] * mu[1] + R[2] * mu[2] + cam.t[0];
    const float pcy = R[3] * mu[0] + R[4] * mu[1] + R[5] * mu[2] + cam.t[1];
    const float pcz = R[6] * mu[0] + R[7] * mu[1] + R[8] * mu[2] + cam.t[2];
    // rotation
    const float qn = sqrtf(qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3]);
    float w = 1.f, x = 0.f, y = 0.f, z = 0.f;
    if (qn > 0.f) { w = qv[0] / qn; x = qv[1] / qn; y = qv[2] / qn; z = qv[3] / qn; }
    float r[9];
    r[0] = 1.f - 2.f * (y * y + z * z); r[1] = 2.f * (x * y - w * z); r[2] = 2.f * (x * z + w * y);
    r[3] = 2.f * (x * y + w * z); r[4] = 1.f - 2.f * (x * x + z * z); r[5] = 2.f * (y * z - w * x);
    r[6] = 2.f * (x * z - w * y); r[7] = 2.f * (y * z + w * x); r[8] = 1.f - 2.f * (x * x + y * y);
    float M[9];
#pragma unroll
    for (int jj = 0; jj < 3; ++jj)
#pragma unroll
      for (int k = 0; k < 3; ++k) M[3 * jj + k] = r[3 * jj + k] * s[k];
    // J at the clamped mean
    const float tx = pcx / pcz, ty = pcy / pcz;
    const int clx = tx > vd.limx ? 1 : (tx < -vd.limx ? -1 : 0);
    const int cly = ty > vd.limy ? 1 : (ty < -vd.limy ? -1 : 0);
    const float xc = clx ? clx * vd.limx * pcz : pcx;
    const float yc = cly ? cly * vd.limy * pcz : pcy;
    const float iz = 1.f / pcz, iz2 = iz * iz;
    const float j00 = cam.fx * iz, j02 = -cam.fx * xc * iz2;
    const float j11 = cam.fy * iz, j12 = -cam.fy * yc * iz2;
    float T0[3], T1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T0[k] = j00 * R[k] + j02 * R[6 + k];
      T1[k] = j11 * R[3 + k] + j12 * R[6 + k];
    }
    float G0[3], G1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      G0[k] = T0[0] * M[k] + T0[1] * M[3 + k] + T0[2] * M[6 + k];
      G1[k] = T1[0] * M[k] + T1[1] * M[3 + k] + T1[2] * M[6 + k];
    }
    // Q from the whitening rows of the forward: Q = (w1 w1^T + w2 w2^T) / kWhiten^2
    const float4 sh4 = a.rec_shape[j];
    const float iw = 1.0f / (kWhiten * kWhiten);
    const float Qa = (sh4.x * sh4.x + sh4.z * sh4.z) * iw;
    const float Qb = (sh4.x * sh4.y + sh4.z * sh4.w) * iw;
    const float Qc = (sh4.y * sh4.y + sh4.w * sh4.w) * iw;
    // dSigma' = -Q dQ Q, dQ symmetric with the off-diagonal gradient split
    const float da = gqa, db = 0.5f * gqb, dc = gqc;
    const float t00 = da * Qa + db * Qb, t01 = da * Qb + db * Qc;
    const float t10 = db * Qa + dc * Qb, t11 = db * Qb + dc * Qc;
    const float dS00 = -(Qa * t00 + Qb * t10);
    const float dS01 = -(Qa * t01 + Qb * t11);
    const float dS11 = -(Qb * t01 + Qc * t11);
    // Sigma' = G G^T + 0.3 I: dG = 2 dSigma' G
    float dG0[3], dG1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dG0[k] = 2.f * (dS00 * G0[k] + dS01 * G1[k]);
      dG1[k] = 2.f * (dS01 * G0[k] + dS11 * G1[k]);
    }
    // G = T M: dT = dG M^T, dM = T^T dG
    float dT0[3], dT1[3], dM[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dT0[k] = dG0[0] * M[3 * k] + dG0[1] * M[3 * k + 1] + dG0[2] * M[3 * k + 2];
      dT1[k] = dG1[0] * M[3 * k] + dG1[1] * M[3 * k + 1] + dG1[2] * M[3 * k + 2];
    }
#pragma unroll
    for (int jj = 0; jj < 3; ++jj)
#pragma unroll
      for (int k = 0; k < 3; ++k) dM[3 * jj + k] = T0[jj] * dG0[k] + T1[jj] * dG1[k];
    // M = Rq diag(s)
    float ds[3] = {0.f, 0.f, 0.f}, dR[9];
#pragma unroll
    for (int jj = 0; jj < 3; ++jj)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ds[k] += dM[3 * jj + k] * r[3 * jj + k];
        dR[3 * jj + k] = dM[3 * jj + k] * s[k];
      }
    float dqn[4];
    dqn[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dqn[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] +
                    w * dR[7] - 2.f * x * dR[8]);
    dqn[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] -
                    w * dR[6] + z * dR[7] - 2.f * y * dR[8]);
    dqn[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] +
                    y * dR[5] + x * dR[6] + y * dR[7]);
    float dq[4] = {0.f, 0.f, 0.f, 0.f};
    if (qn > 0.f) {
      const float dot = dqn[0] * w + dqn[1] * x + dqn[2] * y + dqn[3] * z;
      dq[0] = (dqn[0] - dot * w) / qn;
      dq[1] = (dqn[1] - dot * x) / qn;
      dq[2] = (dqn[2] - dot * y) / qn;
      dq[3] = (dqn[3] - dot * z) / qn;
    }
    // T = J W: dJ = dT W^T (rows of W are the camera axes)
    const float dJ00 = dT0[0] * R[0] + dT0[1] * R[1] + dT0[2] * R[2];
    const float dJ02 = dT0[0] * R[6] + dT0[1] * R[7] + dT0[2] * R[8];
    const float dJ11 = dT1[0] * R[3] + dT1[1] * R[4] + dT1[2] * R[5];
    const float dJ12 = dT1[0] * R[6] + dT1[1] * R[7] + dT1[2] * R[8];
    float dpx = 0.f, dpy = 0.f, dpz = 0.f;
    dpz += -dJ00 * cam.fx * iz2 - dJ11 * cam.fy * iz2 + 2.f * dJ02 * cam.fx * xc * iz2 * iz +
           2.f * dJ12 * cam.fy * yc * iz2 * iz;
    const float dxc = -dJ02 * cam.fx * iz2, dyc = -dJ12 * cam.fy * iz2;
    if (clx) dpz += dxc * clx * vd.limx; else dpx += dxc;
    if (cly) dpz += dyc * cly * vd.limy; else dpy += dyc;
    // 2D mean: u = fx x / z + cx
    dpx += gmx * cam.fx * iz;
    dpy += gmy * cam.fy * iz;
    dpz += -(gmx * cam.fx * pcx + gmy * cam.fy * pcy) * iz2;
    float dmu[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dmu[k] = R[k] * dpx + R[3 + k] * dpy + R[6 + k] * dpz;
    // colour through the SH basis at the view direction
    const float vx = mu[0] - vd.ccx, vy = mu[1] - vd.ccy, vz = mu[2] - vd.ccz;
    const float vn = sqrtf(vx * vx + vy * vy + vz * vz);
    const float ivn = vn > 0.f ? 1.f / vn : 0.f;
    const float dxn = vx * ivn, dyn = vy * ivn, dzn = vz * ivn;
    float Y[16], dY[16][3];
    sh_basis_and_grad(dxn, dyn, dzn, S, Y, dY);
    const float *shc = a.sh + (long long)S * 3 * i;
    float *dsh = a.d_sh + (long long)S * 3 * i;
    float ddir[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float raw = kShOffset;
#pragma unroll
      for (int k = 0; k < S; ++k) raw = fmaf(shc[3 * k + ch], Y[k], raw);
      if (!(raw > 0.f) || gc[ch] == 0.f) continue;
#pragma unroll
      for (int k = 0; k < S; ++k) {
        atomicAdd(&dsh[3 * k + ch], Y[k] * gc[ch]);
        if (k > 0) {
          ddir[0] += shc[3 * k + ch] * dY[k][0] * gc[ch];
          ddir[1] += shc[3 * k + ch] * dY[k][1] * gc[ch];
          ddir[2] += shc[3 * k + ch] * dY[k][2] * gc[ch];
        }
      }
    }
    // per-level opacity / DC of levels 2..L
    if (a.grad_lv) {
      for (int l = 2; l <= a.L; ++l) {
        const float *gl = a.grad_lv + ((long long)(l - 2) * a.max_visible + j) * kGradLv;
        if (gl[0] != 0.f) {
          // a level without its own opacity shares the base one
          if (a.opacity_lv) atomicAdd(&a.d_opac_lv[(long long)(l - 2) * a.n + i], gl[0]);
          else atomicAdd(&a.d_opac[i], gl[0]);
        }
        if (!a.dc_lv) {
          // shared colour: the level's colour gradient goes to the base SH
          for (int ch = 0; ch < 3; ++ch) {
            const float g = gl[1 + ch];
            if (g == 0.f) continue;
            float raw = kShOffset;
            for (int k = 0; k < S; ++k) raw = fmaf(shc[3 * k + ch], Y[k], raw);
            if (!(raw > 0.f)) continue;
            for (int k = 0; k < S; ++k) {
              atomicAdd(&dsh[3 * k + ch], Y[k] * g);
              if (k > 0)
                for (int e = 0; e < 3; ++e) ddir[e] += shc[3 * k + ch] * dY[k][e] * g;
            }
          }
          continue;
        }
        for (int ch = 0; ch < 3; ++ch) {
          const float g = gl[1 + ch];
          if (g == 0.f) continue;
          float raw = kShOffset + kY00b * a.dc_lv[((long long)(l - 2) * a.n + i) * 3 + ch];
          for (int k = 1; k < S; ++k) raw = fmaf(shc[3 * k + ch], Y[k], raw);
          if (!(raw > 0.f)) continue;
          atomicAdd(&a.d_dc_lv[((long long)(l - 2) * a.n + i) * 3 + ch], kY00b * g);
          for (int k = 1; k < S; ++k) {
            atomicAdd(&dsh[3 * k + ch], Y[k] * g);
            for (int e = 0; e < 3; ++e) ddir[e] += shc[3 * k + ch] * dY[k][e] * g;
          }
        }
      }
    }
    const float dd = ddir[0] * dxn + ddir[1] * dyn + ddir[2] * dzn;
    dmu[0] += (ddir[0] - dd * dxn) * ivn;
    dmu[1] += (ddir[1] - dd * dyn) * ivn;
    dmu[2] += (ddir[2] - dd * dzn) * ivn;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicAdd(&a.d_means[3 * i + k], dmu[k]);
      atomicAdd(&a.d_scales[3 * i + k], ds[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(&a.d_quats[4 * i + k], dq[k]);
    if (gop != 0.f) atomicAdd(&a.d_opac[i], gop);
  }
}

template <int B>
static void launch_rb(const BwdArgs &a, bool fov, bool mv, long long tiles, cudaStream_t s) {
  if (!fov) k_render_bwd_plain<B><<<(unsigned)tiles, B * B / 2, 0, s>>>(a);
  else if (!mv) k_render_bwd_fov<B><<<(unsigned)tiles, B * B / 2, 0, s>>>(a);
  else k_render_bwd<B, true, true><<<(unsigned)tiles, B * B, 0, s>>>(a);
}

cudaError_t launch_backward(const gs_plan *p, void *ws, const float *dL, const float *T,
                            const int32_t *last, const float bg[3], float *d_means,
                            float *d_scales, float *d_quats, float *d_opac, float *d_sh,
                            float *d_opac_lv, float *d_dc_lv, cudaStream_t s) {
  const long long n = p->n;
  const int S = (p->sh_degree + 1) * (p->sh_degree + 1);
  const bool fov = p->last_fov != 0;
  const bool mv = fov && p->fov_mv;
  const int L = fov ? p->fov.n_levels : 1;
  cudaError_t e;
  if (n > 0) {
    if ((e = cudaMemsetAsync(d_means, 0, 12 * n, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_scales, 0, 12 * n, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_quats, 0, 16 * n, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_opac, 0, 4 * n, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_sh, 0, 12 * (size_t)S * n, s)) != cudaSuccess) return e;
    if (mv && d_opac_lv && (e = cudaMemsetAsync(d_opac_lv, 0, 4 * (size_t)(L - 1) * n, s)) != cudaSuccess) return e;
    if (mv && d_dc_lv && (e = cudaMemsetAsync(d_dc_lv, 0, 12 * (size_t)(L - 1) * n, s)) != cudaSuccess) return e;
  }
  if (n == 0 || p->tiles_total == 0) return cudaGetLastError();
  Hdr *hdr = region<Hdr>(p, ws, R_HDR);
  float *grad_item = region<float>(p, ws, R_GRAD_ITEM);
  float *grad_lv = mv ? region<float>(p, ws, R_GRAD_LV) : nullptr;
  if ((e = cudaMemsetAsync(grad_item, 0, sizeof(float) * kGradItem * (size_t)p->max_visible, s)) != cudaSuccess) return e;
  if (grad_lv && (e = cudaMemsetAsync(grad_lv, 0, sizeof(float) * kGradLv * (size_t)(L - 1) * p->max_visible, s)) != cudaSuccess) return e;
  BwdArgs a = {};
  a.views = region<ViewDev>(p, ws, R_VIEWS);
  a.V = p->V;
  a.n = n;
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
  a.opac = p->scene.opacities;
  a.L = L;
  a.band = fov ? p->fov.band_px : 0.f;
  a.mmfr = fov && (p->flags & GS_FLAG_MULTI_MODEL) ? 1 : 0;
  a.opacity_lv = mv ? p->fov.opacity_lv : nullptr;
  a.dc_lv = mv ? p->fov.dc_lv : nullptr;
  a.bg0 = bg[0]; a.bg1 = bg[1]; a.bg2 = bg[2];
  a.dL = dL;
  a.T = T;
  a.last = last;
  a.grad_item = grad_item;
  a.grad_lv = grad_lv;
  a.max_visible = p->max_visible;
  if (p->tile == 16) launch_rb<16>(a, fov, mv, p->tiles_total, s);
  else launch_rb<8>(a, fov, mv, p->tiles_total, s);

  PBwdArgs b = {};
  b.n = n;
  b.S = S;
  b.means = p->scene.means; b.scales = p->scene.scales; b.quats = p->scene.quats;
  b.opac = p->scene.opacities; b.sh = p->scene.sh;
  b.cams = p->cams;
  b.views = a.views;
  b.n_items = &hdr->n_items;
  b.rec_depth = region<uint32_t>(p, ws, R_REC_DEPTH);
  b.max_visible = p->max_visible;
  b.rec_gid = a.rec_gid;
  b.rec_view = region<uint32_t>(p, ws, R_REC_VIEW);
  b.rec_shape = a.rec_shape;
  b.grad_item = grad_item;
  b.grad_lv = grad_lv;
  b.L = L;
  b.opacity_lv = a.opacity_lv;
  b.dc_lv = a.dc_lv;
  b.d_means = d_means; b.d_scales = d_scales; b.d_quats = d_quats; b.d_opac = d_opac;
  b.d_sh = d_sh; b.d_opac_lv = d_opac_lv; b.d_dc_lv = d_dc_lv;
  const int grid = p->num_sms > 0 ? p->num_sms * 8 : 1024;
  switch (S) {
    case 1: k_project_bwd<1><<<grid, 128, 0, s>>>(b); break;
    case 4: k_project_bwd<4><<<grid, 128, 0, s>>>(b); break;
    case 9: k_project_bwd<9><<<grid, 128, 0, s>>>(b); break;
    default: k_project_bwd<16><<<grid, 128, 0, s>>>(b); break;
  }
  return cudaGetLastError();
}

}  // namespace gs
