// k_sort.cu -- Sorting stage (Sec. 2.1 "Sorting": per tile, the intersecting
// ellipses ordered by depth, closest first).
//
// The per-tile depth order is produced by two stable LSD radix sorts:
//   1. the visible (view, point) items by the FP32 bits of camera depth
//      (ties keep item order, i.e. point index inside a view);
//   2. the (tile, item) pairs, emitted in that depth order, by tile id.
// Together they order the pairs by (tile, depth, point index), the same
// order as one stable sort of (tile << 32 | depth) keys.
//
// Each radix pass is a single "onesweep" kernel: persistent blocks take
// 4096-key partitions by atomic ticket, rank digits inside each warp with
// __match_any_sync, publish per-digit partition counts and look back over
// their predecessors (decoupled look-back, bounded spin) to get global
// positions, then scatter.  A pass whose digit is the same for all keys is
// skipped on the device.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gs_internal.cuh"
#include "lookback.cuh"

namespace gs {

struct SortArgs {
  const uint32_t *first_keys;        // input keys (read by the first executed pass)
  const uint32_t *first_vals;        // input values, or null: values = key index
  uint32_t *keys[2];                 // ping-pong buffers
  uint32_t *vals[2];
  const unsigned long long *count;   // device-side number of keys
  long long capacity;                // keys beyond are ignored
  uint32_t *sel;                     // out: buffer index holding the result
  uint32_t *hist;                    // [4][256] digit histograms -> offsets
  uint32_t *skip;                    // [4] pass skipped (constant digit)
  uint32_t *tickets;                 // [4] partition tickets
  unsigned long long *lb;            // [2][max_parts][256] look-back slots
  long long max_parts;
  int passes;
  int digit_bits;                    // bits per pass (<= 8)
  int no_skip;                       // run every pass (fixed buffer parity)
  uint32_t *status;
};

__device__ __forceinline__ uint32_t sort_n(const SortArgs &a) {
  unsigned long long n = *a.count;
  if ((long long)n > a.capacity) n = (unsigned long long)a.capacity;
  return (uint32_t)n;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---- histograms of every pass in one read; also resets tickets and the
// first look-back buffer -------------------------------------------------
__global__ void __launch_bounds__(256) k_hist(SortArgs a) {
  __shared__ uint32_t sh[4][256];
  const uint32_t n = sort_n(a);
  for (int q = threadIdx.x; q < 4 * 256; q += blockDim.x) (&sh[0][0])[q] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // warp-uniform trip count so that __match_any_sync sees the full warp
  const long long start = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long iters = ((long long)n + stride - 1) / stride;
  for (long long it = 0; it < iters; ++it) {
    long long idx = start + it * stride;
    bool valid = idx < (long long)n;
    uint32_t key = valid ? a.first_keys[idx] : 0u;
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    const uint32_t dmask = (1u << a.digit_bits) - 1u;
    for (int p = 0; p < a.passes; ++p) {
      const uint32_t d = (key >> (a.digit_bits * p)) & dmask;
      // a warp whose valid keys share the digit adds once (common for the
      // high bytes of depth keys); otherwise every lane adds
      const uint32_t d0 = __shfl_sync(0xffffffffu, d, __ffs(vmask | 1u) - 1);
      if (__all_sync(0xffffffffu, !valid || d == d0)) {
        if (lane == 0 && vmask) atomicAdd(&sh[p][d0], (uint32_t)__popc(vmask));
      } else if (valid) {
        atomicAdd(&sh[p][d], 1u);
      }
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < a.passes * 256; q += blockDim.x) {
    uint32_t c = (&sh[0][0])[q];
    if (c) atomicAdd(&a.hist[q], c);
  }
  // reset look-back buffer 0 for the partitions this sort will use
  const long long nparts = ((long long)n + kSortPart - 1) / kSortPart;
  for (long long q = start; q < nparts * 256; q += stride) a.lb[q] = 0ull;
  if (blockIdx.x == 0 && threadIdx.x < 4) a.tickets[threadIdx.x] = 0u;
}

// exclusive scan of each pass's histogram; constant-digit passes skipped
__global__ void __launch_bounds__(256) k_hist_scan(SortArgs a) {
  __shared__ uint32_t s_w[8];
  const uint32_t n = sort_n(a);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  int executed = 0;
  // an index-generating sort must run at least one pass to write its values
  const bool force_first = a.first_vals == nullptr;
  for (int p = 0; p < a.passes; ++p) {
    uint32_t c = a.hist[p * 256 + t];
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    uint32_t woff = 0;
    for (int q = 0; q < w; ++q) woff += s_w[q];
    a.hist[p * 256 + t] = woff + incl - c;
    int constant = __syncthreads_or(c == n);
    bool sk = (constant || n == 0) && !(force_first && executed == 0 && p == a.passes - 1) &&
              !a.no_skip;
    if (t == 0) a.skip[p] = sk ? 1u : 0u;
    executed += sk ? 0 : 1;
    __syncthreads();
  }
  if (t == 0) *a.sel = (uint32_t)(executed & 1);
}

// ---- one onesweep pass -----------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) k_onesweep(SortArgs a, int pass) {
  __shared__ uint32_t s_wh[kSortThreads / 32][256];
  __shared__ uint32_t s_base[256];
  __shared__ uint32_t s_dstart[256];
  __shared__ uint32_t s_key[kSortPart];
  __shared__ uint32_t s_val[kSortPart];
  __shared__ uint32_t s_part;
  __shared__ uint32_t s_wsum[kSortThreads / 32];
  const uint32_t n = sort_n(a);
  const long long nparts = ((long long)n + kSortPart - 1) / kSortPart;
  unsigned long long *lb_next = a.lb + (long long)((pass + 1) & 1) * a.max_parts * 256;
  if (a.skip[pass]) {
    // keep the next pass's look-back buffer clean even though this one idles
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nparts * 256;
         q += stride)
      lb_next[q] = 0ull;
    return;
  }
  unsigned long long *lb_cur = a.lb + (long long)(pass & 1) * a.max_parts * 256;
  int before = 0;
  for (int p = 0; p < pass; ++p) before += a.skip[p] ? 0 : 1;
  const uint32_t *kin = before == 0 ? a.first_keys : a.keys[before & 1];
  const uint32_t *vin = before == 0 ? a.first_vals : a.vals[before & 1];
  uint32_t *kout = a.keys[(before + 1) & 1];
  uint32_t *vout = a.vals[(before + 1) & 1];
  const bool iota = vin == nullptr;
  const int shift = a.digit_bits * pass;
  const uint32_t dmask = (1u << a.digit_bits) - 1u;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t ltmask = lanemask_lt();
  const uint32_t *goff = a.hist + pass * 256;

  for (;;) {
    if (tid == 0) s_part = atomicAdd(&a.tickets[pass], 1u);
    for (int q = tid; q < (kSortThreads / 32) * 256; q += kSortThreads) (&s_wh[0][0])[q] = 0u;
    __syncthreads();
    const uint32_t part = s_part;
    if ((long long)part >= nparts) break;
    const long long wbase = (long long)part * kSortPart + warp * (32 * kSortItems);
    uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      long long idx = wbase + k * 32 + lane;
      bool valid = idx < (long long)n;
      key[k] = valid ? kin[idx] : 0u;
      val[k] = valid ? (iota ? (uint32_t)idx : vin[idx]) : 0u;
    }
    // warp-level stable ranking (original order = (k, lane))
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      long long idx = wbase + k * 32 + lane;
      bool valid = idx < (long long)n;
      uint32_t d = (key[k] >> shift) & dmask;
      uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 0x100u);
      uint32_t before_w = valid ? s_wh[warp][d] : 0u;
      rank[k] = before_w + __popc(peers & ltmask);
      __syncwarp();
      if (valid && (__ffs(peers) - 1) == lane) s_wh[warp][d] = before_w + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // per digit: warp offsets inside the partition, then look-back
    {
      const int d = tid;  // kSortThreads == 256 digits
      uint32_t tot = 0;
#pragma unroll
      for (int w = 0; w < kSortThreads / 32; ++w) {
        uint32_t c = s_wh[w][d];
        s_wh[w][d] = tot;
        tot += c;
      }
      unsigned long long *slot = lb_cur + (long long)part * 256 + d;
      unsigned long long excl = 0;
      if (part == 0) {
        st_release_u64(slot, kFlagPre | tot);
      } else {
        st_release_u64(slot, kFlagAgg | tot);
        // walk back kLbVec slots per step: the loads of one step are
        // independent, so the chain costs one memory latency per kLbVec
        // predecessors
        constexpr int kLbVec = 16;
        long long q = (long long)part - 1;
        int spins = 0;
        bool done = false;
        while (!done && q >= 0) {
          unsigned long long wv[kLbVec];
#pragma unroll
          for (int v = 0; v < kLbVec; ++v)
            wv[v] = q - v >= 0 ? ld_relaxed_u64(lb_cur + (q - v) * 256 + d) : (kFlagPre | 0ull);
          int used = 0;
#pragma unroll
          for (int v = 0; v < kLbVec; ++v) {
            if (done || used < v) continue;       // stopped earlier in this step
            const unsigned long long f = wv[v] >> 62;
            if (f == 0ull) continue;               // not ready: retry from here
            excl += wv[v] & kValMask;
            if (f == 2ull) done = true;
            used = v + 1;
          }
          q -= used;
          if (!done && used < kLbVec) {
            if (++spins > kSpinLimit) { set_status(a.status, GS_ERR_TIMEOUT); break; }
            __nanosleep(20);
          }
        }
        st_release_u64(slot, kFlagPre | (excl + tot));
      }
      s_base[d] = goff[d] + (uint32_t)excl;
      lb_next[(long long)part * 256 + d] = 0ull;
      // start of digit d inside the partition (block exclusive scan of tot)
      uint32_t incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (lane == 31) s_wsum[warp] = incl;
      __syncthreads();
      uint32_t wofs = 0;
#pragma unroll
      for (int w = 0; w < kSortThreads / 32; ++w) wofs += w < warp ? s_wsum[w] : 0u;
      s_dstart[d] = wofs + incl - tot;
    }
    __syncthreads();
    // stage the partition in digit order, then write runs of equal digits
    // to consecutive global addresses
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      long long idx = wbase + k * 32 + lane;
      if (idx < (long long)n) {
        uint32_t d = (key[k] >> shift) & dmask;
        uint32_t lp = s_dstart[d] + s_wh[warp][d] + rank[k];
        s_key[lp] = key[k];
        s_val[lp] = val[k];
      }
    }
    __syncthreads();
    const long long pbase = (long long)part * kSortPart;
    const uint32_t pcount = (uint32_t)min((long long)kSortPart, (long long)n - pbase);
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      const uint32_t lp = (uint32_t)(k * kSortThreads + tid);
      if (lp < pcount) {
        const uint32_t kk = s_key[lp];
        const uint32_t d = (kk >> shift) & dmask;
        const uint32_t dst = s_base[d] + (lp - s_dstart[d]);
        if (dst < n) {
          kout[dst] = kk;
          vout[dst] = s_val[lp];
        }
      }
    }
    __syncthreads();
  }
}

static int g_sort_blocks = 0;
static int g_stream_blocks = 0;   // grid of the streaming kernels (emit, offsets, ranges, hist)

static cudaError_t run_sort(const SortArgs &a, cudaStream_t s, bool hist_done = false) {
  if (g_sort_blocks == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_onesweep, kSortThreads, 0);
    g_sort_blocks = sms * (per > 0 ? per : 1);
    g_stream_blocks = sms * 8;
  }
  if (!hist_done) k_hist<<<g_stream_blocks, 256, 0, s>>>(a);
  k_hist_scan<<<1, 256, 0, s>>>(a);
  for (int p = 0; p < a.passes; ++p) k_onesweep<<<g_sort_blocks, kSortThreads, 0, s>>>(a, p);
  return cudaGetLastError();
}

// ---- exclusive scan of pair counts in depth order -> emit offsets --------
struct ScanArgs {
  const uint32_t *sorted_items[2];
  const uint32_t *sel;
  const uint32_t *count;            // rec_count (by item)
  const unsigned long long *n_items;
  long long capacity;
  uint32_t *offsets;
  unsigned long long *slots;
  uint32_t *ticket;
  unsigned long long *n_pairs;
  uint32_t *status;
};

__global__ void __launch_bounds__(256) k_offsets(ScanArgs a) {
  __shared__ uint32_t s_part;
  __shared__ unsigned long long s_w[8];
  __shared__ unsigned long long s_base;
  unsigned long long nn = *a.n_items;
  const uint32_t n = (uint32_t)((long long)nn > a.capacity ? a.capacity : (long long)nn);
  const long long nparts = ((long long)n + kSortPart - 1) / kSortPart;
  const uint32_t *items = a.sorted_items[*a.sel];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    if (tid == 0) s_part = atomicAdd(a.ticket, 1u);
    __syncthreads();
    const uint32_t part = s_part;
    if ((long long)part >= nparts) break;
    const long long base = (long long)part * kSortPart + (long long)tid * 16;
    unsigned long long c[16];
    unsigned long long tsum = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      long long idx = base + k;
      c[k] = idx < (long long)n ? a.count[items[idx]] : 0ull;
      tsum += c[k];
    }
    unsigned long long incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    unsigned long long woff = 0, total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      if (w < warp) woff += s_w[w];
      total += s_w[w];
    }
    if (warp == 0) {
      unsigned long long ex = lookback_single_warp(a.slots, part, total, a.status);
      if (lane == 0) {
        s_base = ex;
        if ((long long)part == nparts - 1) *a.n_pairs = ex + total;
      }
    }
    __syncthreads();
    unsigned long long run = s_base + woff + incl - tsum;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      long long idx = base + k;
      if (idx < (long long)n) a.offsets[idx] = (uint32_t)(run > 0xffffffffull ? 0xffffffffull : run);
      run += c[k];
    }
    __syncthreads();
  }
}

// ---- emit (tile, item) pairs in depth order ------------------------------
struct EmitArgs {
  const uint32_t *sorted_items[2];
  const uint32_t *sel;
  const unsigned long long *n_items;
  long long item_capacity;
  const uint32_t *offsets;
  const uint32_t *count;
  const uint2 *rect;
  const uint32_t *view;
  const ViewDev *views;
  const uint8_t *tile_level;
  const uint8_t *rec_m;
  const unsigned long long *n_pairs;
  long long pair_capacity;
  uint32_t *pkey, *pval;
  uint32_t *bigq;                    // queue of items with more than kBigItem tiles
  uint32_t *big_count, *big_ticket;
  uint32_t *hist;                    // pair sort histograms [passes][256]
  unsigned long long *lb;            // pair sort look-back buffer 0
  int passes, digit_bits;
  uint32_t *status;
};

// Warp-synchronous: each lane takes one item of a 32-item group.  The
// group's pairs occupy one contiguous output range; when it holds at most
// kStage pairs they are assembled in shared memory (small items by their own
// lane, large ones by the whole warp) and written back with coalesced
// stores, the pair sort's digit histograms being taken during that flush.
// Wider groups write directly.  The kernel also clears the pair sort's
// first look-back buffer, so no separate pass reads the keys.
constexpr uint32_t kSmallItem = 8;
constexpr uint32_t kBigItem = 64;   // larger items go to k_emit_big
constexpr int kStage = 768;
constexpr int kEmitThreads = 128;

__device__ __forceinline__ void hist_add_warp(uint32_t (*sh)[256], bool on, uint32_t t,
                                              int passes, int bits, uint32_t dmask, int lane) {
  const uint32_t m = __ballot_sync(0xffffffffu, on);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  for (int p = 0; p < passes; ++p) {
    const uint32_t dg = (t >> (bits * p)) & dmask;
    const uint32_t d0 = __shfl_sync(0xffffffffu, dg, leader);
    if (__all_sync(0xffffffffu, !on || dg == d0)) {
      if (lane == leader) atomicAdd(&sh[p][d0], (uint32_t)__popc(m));
    } else if (on) {
      atomicAdd(&sh[p][dg], 1u);
    }
  }
}

__global__ void __launch_bounds__(kEmitThreads) k_emit(EmitArgs a) {
  __shared__ uint32_t sh[4][256];
  __shared__ uint32_t s_t[kEmitThreads / 32][kStage];
  __shared__ uint32_t s_v[kEmitThreads / 32][kStage];
  for (int q = threadIdx.x; q < 4 * 256; q += blockDim.x) (&sh[0][0])[q] = 0u;
  __syncthreads();
  unsigned long long nn = *a.n_items;
  const long long n = (long long)nn > a.item_capacity ? a.item_capacity : (long long)nn;
  const uint32_t *items = a.sorted_items[*a.sel];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const uint32_t ltmask = (1u << lane) - 1u;
  const uint32_t dmask = (1u << a.digit_bits) - 1u;
  if (blockIdx.x == 0 && threadIdx.x == 0 && (long long)*a.n_pairs > a.pair_capacity)
    set_status(a.status, GS_ERR_CAPACITY);
  const long long warps = (long long)gridDim.x * (blockDim.x / 32);
  const long long wid = (long long)blockIdx.x * (blockDim.x / 32) + wl;
  uint32_t *st = s_t[wl], *sv = s_v[wl];
  for (long long base = wid * 32; base < n; base += warps * 32) {
    const long long k = base + lane;
    const bool valid = k < n;
    uint32_t j = 0, cnt = 0, off = 0, view = 0;
    uint2 r = make_uint2(0u, 0u);
    if (valid) {
      j = items[k];
      off = a.offsets[k];
      cnt = a.count[j];
      r = a.rect[j];
      view = a.view[j];
    }
    // items with more than kBigItem tiles are queued for k_emit_big, whose
    // warps take them one at a time (they cluster in depth order and would
    // otherwise leave a few warps with most of the work)
    const bool huge = valid && cnt > kBigItem;
    const uint32_t hb = __ballot_sync(0xffffffffu, huge);
    const bool any_huge = hb != 0u;
    if (any_huge) {
      // one queue reservation per warp
      uint32_t base = 0;
      if (lane == __ffs(hb) - 1) base = atomicAdd(a.big_count, (uint32_t)__popc(hb));
      base = __shfl_sync(0xffffffffu, base, __ffs(hb) - 1);
      if (huge) a.bigq[base + __popc(hb & ltmask)] = (uint32_t)k;
    }
    // the group's output range [g0, g1)
    const uint32_t g0 = __shfl_sync(0xffffffffu, off, 0);
    const uint32_t last = 31 - __clz(__ballot_sync(0xffffffffu, valid));
    const uint32_t g1 = __shfl_sync(0xffffffffu, off + cnt, last);
    const bool staged = !any_huge && g1 - g0 <= (uint32_t)kStage;
    // small items: one lane each
    if (valid && cnt <= kSmallItem && cnt > 0) {
      const ViewDev &vd = a.views[view];
      const int x0 = r.x & 0xffff, x1 = r.x >> 16, y0 = r.y & 0xffff, y1 = r.y >> 16;
      const uint8_t m = a.tile_level ? a.rec_m[j] : 0;
      long long o = off;
      for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) {
          const long long t = vd.tile_base + (long long)y * vd.tx + x;
          if (a.tile_level && a.tile_level[t] > m) continue;
          if (staged) {
            st[o - g0] = (uint32_t)t;
            sv[o - g0] = j;
          } else if (o < a.pair_capacity) {
            a.pkey[o] = (uint32_t)t;
            a.pval[o] = j;
            for (int p = 0; p < a.passes; ++p)
              atomicAdd(&sh[p][((uint32_t)t >> (a.digit_bits * p)) & dmask], 1u);
          }
          ++o;
        }
    }
    // large items: the whole warp, one item at a time
    uint32_t big = __ballot_sync(0xffffffffu, valid && cnt > kSmallItem && cnt <= kBigItem);
    while (big) {
      const int src = __ffs(big) - 1;
      big &= big - 1;
      const uint32_t bj = __shfl_sync(0xffffffffu, j, src);
      const uint32_t boff = __shfl_sync(0xffffffffu, off, src);
      const uint32_t rx = __shfl_sync(0xffffffffu, r.x, src);
      const uint32_t ry = __shfl_sync(0xffffffffu, r.y, src);
      const uint32_t bview = __shfl_sync(0xffffffffu, view, src);
      const ViewDev &vd = a.views[bview];
      const int x0 = rx & 0xffff, x1 = rx >> 16, y0 = ry & 0xffff, y1 = ry >> 16;
      const int w = x1 - x0 + 1;
      const int area = w * (y1 - y0 + 1);
      const uint8_t m = a.tile_level ? a.rec_m[bj] : 0;
      long long run = boff;
      for (int l0 = 0; l0 < area; l0 += 32) {
        const int l = l0 + lane;
        bool kept = l < area;
        long long t = 0;
        if (kept) {
          t = vd.tile_base + (long long)(y0 + l / w) * vd.tx + (x0 + l % w);
          if (a.tile_level && a.tile_level[t] > m) kept = false;
        }
        // every lane takes part in the ballots (never inside && or ?:)
        const uint32_t b = __ballot_sync(0xffffffffu, kept);
        const long long o = run + __popc(b & ltmask);
        if (staged) {
          if (kept) {
            st[o - g0] = (uint32_t)t;
            sv[o - g0] = bj;
          }
        } else {
          const bool wr = kept && o < a.pair_capacity;
          if (wr) {
            a.pkey[o] = (uint32_t)t;
            a.pval[o] = bj;
          }
          hist_add_warp(sh, wr, (uint32_t)t, a.passes, a.digit_bits, dmask, lane);
        }
        run += __popc(b);
      }
    }
    // coalesced flush of a staged group
    if (staged) {
      __syncwarp();
      for (uint32_t l0 = 0; l0 < g1 - g0; l0 += 32) {
        const uint32_t l = l0 + lane;
        const long long o = (long long)g0 + l;
        const bool wr = l < g1 - g0 && o < a.pair_capacity;
        const uint32_t t = wr ? st[l] : 0u;
        if (wr) {
          a.pkey[o] = t;
          a.pval[o] = sv[l];
        }
        hist_add_warp(sh, wr, t, a.passes, a.digit_bits, dmask, lane);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < a.passes * 256; q += blockDim.x) {
    const uint32_t c = (&sh[0][0])[q];
    if (c) atomicAdd(&a.hist[q], c);
  }
  // clear the pair sort's first look-back buffer for the partitions it uses
  unsigned long long kk = *a.n_pairs;
  const long long K = (long long)kk > a.pair_capacity ? a.pair_capacity : (long long)kk;
  const long long nparts = (K + kSortPart - 1) / kSortPart;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nparts * 256;
       q += (long long)gridDim.x * blockDim.x)
    a.lb[q] = 0ull;
}

// Items with more than kBigItem tiles: the warps of the grid stride over the
// queue (no shared ticket to contend on) and write each item's tiles 32 at a
// time (ballot prefix for the kept ones).
__global__ void __launch_bounds__(256) k_emit_big(EmitArgs a) {
  __shared__ uint32_t sh[4][256];
  for (int q = threadIdx.x; q < 4 * 256; q += blockDim.x) (&sh[0][0])[q] = 0u;
  __syncthreads();
  const uint32_t nbig = *a.big_count;
  const uint32_t *items = a.sorted_items[*a.sel];
  const int lane = threadIdx.x & 31;
  const uint32_t ltmask = (1u << lane) - 1u;
  const uint32_t dmask = (1u << a.digit_bits) - 1u;
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  for (uint32_t qi = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); qi < nbig; qi += warps) {
    const uint32_t k = a.bigq[qi];
    const uint32_t j = items[k];
    const uint32_t off = a.offsets[k];
    const uint2 r = a.rect[j];
    const ViewDev &vd = a.views[a.view[j]];
    const int x0 = r.x & 0xffff, x1 = r.x >> 16, y0 = r.y & 0xffff, y1 = r.y >> 16;
    const int w = x1 - x0 + 1;
    const uint8_t m = a.tile_level ? a.rec_m[j] : 0;
    long long run = off;
    // row by row, 32 tiles of a row at a time (no division per tile)
    for (int y = y0, x = 0; y <= y1; x += 32) {
      if (x >= w) {
        x = -32;
        ++y;
        continue;
      }
      const int xx = x + lane;
      bool kept = xx < w;
      long long t = 0;
      if (kept) {
        t = vd.tile_base + (long long)y * vd.tx + (x0 + xx);
        if (a.tile_level && a.tile_level[t] > m) kept = false;
      }
      const uint32_t b = __ballot_sync(0xffffffffu, kept);
      const long long o = run + __popc(b & ltmask);
      const bool wr = kept && o < a.pair_capacity;
      if (wr) {
        a.pkey[o] = (uint32_t)t;
        a.pval[o] = j;
      }
      hist_add_warp(sh, wr, (uint32_t)t, a.passes, a.digit_bits, dmask, lane);
      run += __popc(b);
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < a.passes * 256; q += blockDim.x) {
    const uint32_t c = (&sh[0][0])[q];
    if (c) atomicAdd(&a.hist[q], c);
  }
}

// ---- per-tile ranges ------------------------------------------------------
__global__ void __launch_bounds__(256) k_ranges(const uint32_t *key_a, const uint32_t *key_b,
                                                const uint32_t *sel,
                                                const unsigned long long *n_pairs,
                                                long long capacity, uint2 *ranges) {
  unsigned long long nn = *n_pairs;
  const long long n = (long long)nn > capacity ? capacity : (long long)nn;
  const uint32_t *key = *sel ? key_b : key_a;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    const uint32_t t = key[p];
    if (p == 0 || key[p - 1] != t) ranges[t].x = (uint32_t)p;
    if (p == n - 1 || key[p + 1] != t) ranges[t].y = (uint32_t)(p + 1);
  }
}

cudaError_t launch_bin_sort(const gs_plan *p, void *ws, cudaStream_t s) {
  Hdr *hdr = region<Hdr>(p, ws, R_HDR);
  cudaError_t e;
  // histograms and tickets of this stage start from zero (ticket 0 belongs
  // to the projection)
  e = cudaMemsetAsync(&hdr->hist[0][0][0], 0, sizeof(hdr->hist), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&hdr->ticket[1], 0, sizeof(hdr->ticket) - sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const long long off_parts = (p->max_visible + kSortPart - 1) / kSortPart;
  e = cudaMemsetAsync(region<unsigned long long>(p, ws, R_SCAN), 0,
                      sizeof(unsigned long long) * (size_t)off_parts, s);
  if (e != cudaSuccess) return e;
  if (p->n == 0) {
    // nothing visible: empty ranges
    e = cudaMemsetAsync(region<uint2>(p, ws, R_RANGES), 0, p->bytes[R_RANGES], s);
    return e;
  }
  const long long max_parts =
      ((p->max_visible > p->max_pairs ? p->max_visible : p->max_pairs) + kSortPart - 1) / kSortPart;
  // 1. depth sort of the visible items
  SortArgs d = {};
  d.first_keys = region<uint32_t>(p, ws, R_REC_DEPTH);
  d.first_vals = nullptr;
  d.keys[0] = region<uint32_t>(p, ws, R_DKEY_A);
  d.keys[1] = region<uint32_t>(p, ws, R_DKEY_B);
  d.vals[0] = region<uint32_t>(p, ws, R_DVAL_A);
  d.vals[1] = region<uint32_t>(p, ws, R_DVAL_B);
  d.count = &hdr->n_items;          // every slot; invisible ones sort last
  d.capacity = p->max_visible;
  d.sel = &hdr->sel_depth;
  d.hist = &hdr->hist[0][0][0];
  d.skip = &hdr->skip[0];
  d.tickets = &hdr->ticket[1];
  d.lb = region<unsigned long long>(p, ws, R_LOOKBACK);
  d.max_parts = max_parts;
  d.passes = 4;
  d.digit_bits = 8;
  d.status = &hdr->status;
  e = run_sort(d, s);
  if (e != cudaSuccess) return e;
  // 2. pair offsets in depth order
  ScanArgs sa = {};
  sa.sorted_items[0] = d.vals[0];
  sa.sorted_items[1] = d.vals[1];
  sa.sel = &hdr->sel_depth;
  sa.count = region<uint32_t>(p, ws, R_REC_COUNT);
  sa.n_items = &hdr->n_visible;
  sa.capacity = p->max_visible;
  sa.offsets = region<uint32_t>(p, ws, R_OFFSETS);
  sa.slots = region<unsigned long long>(p, ws, R_SCAN);
  sa.ticket = &hdr->ticket[9];
  sa.n_pairs = &hdr->n_pairs;
  sa.status = &hdr->status;
  k_offsets<<<g_stream_blocks, 256, 0, s>>>(sa);
  // 3. emit pairs (+ the pair sort's histograms)
  // digit width: the requested one, else the balanced width of the fewest
  // passes of at most 8 bits
  const int want = p->radix_bits > 0 ? p->radix_bits : 8;
  int pair_passes = (p->tile_bits + want - 1) / want;
  if (pair_passes > 4) pair_passes = 4;   // histogram storage holds four passes
  const int pair_bits = (p->tile_bits + pair_passes - 1) / pair_passes;
  EmitArgs ea = {};
  ea.sorted_items[0] = d.vals[0];
  ea.sorted_items[1] = d.vals[1];
  ea.sel = &hdr->sel_depth;
  ea.n_items = &hdr->n_visible;
  ea.item_capacity = p->max_visible;
  ea.offsets = sa.offsets;
  ea.count = sa.count;
  ea.rect = region<uint2>(p, ws, R_REC_RECT);
  ea.view = region<uint32_t>(p, ws, R_REC_VIEW);
  ea.views = region<ViewDev>(p, ws, R_VIEWS);
  ea.tile_level = p->has_fov ? region<uint8_t>(p, ws, R_TILE_LEVEL) : nullptr;
  ea.rec_m = p->has_fov ? region<uint8_t>(p, ws, R_REC_M) : nullptr;
  ea.n_pairs = &hdr->n_pairs;
  ea.pair_capacity = p->max_pairs;
  ea.pkey = region<uint32_t>(p, ws, R_PKEY_A);
  ea.pval = region<uint32_t>(p, ws, R_PVAL_A);
  ea.hist = &hdr->hist[1][0][0];
  ea.lb = d.lb;
  ea.passes = pair_passes;
  ea.digit_bits = pair_bits;
  ea.status = &hdr->status;
  ea.bigq = region<uint32_t>(p, ws, R_BIGQ);
  ea.big_count = &hdr->big_count;
  ea.big_ticket = &hdr->big_ticket;
  e = cudaMemsetAsync(&hdr->big_count, 0, 2 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  k_emit<<<2 * g_stream_blocks, kEmitThreads, 0, s>>>(ea);
  k_emit_big<<<g_stream_blocks, 256, 0, s>>>(ea);
  // 4. stable sort of the pairs by tile
  SortArgs t = {};
  t.first_keys = ea.pkey;
  t.first_vals = ea.pval;
  t.keys[0] = ea.pkey;
  t.keys[1] = region<uint32_t>(p, ws, R_PKEY_B);
  t.vals[0] = ea.pval;
  t.vals[1] = region<uint32_t>(p, ws, R_PVAL_B);
  t.count = &hdr->n_pairs;
  t.capacity = p->max_pairs;
  t.sel = &hdr->sel_pair;
  t.hist = &hdr->hist[1][0][0];
  t.skip = &hdr->skip[4];
  t.tickets = &hdr->ticket[5];
  t.lb = d.lb;
  t.max_parts = max_parts;
  t.passes = pair_passes;
  t.digit_bits = pair_bits;
  t.status = &hdr->status;
  e = run_sort(t, s, /*hist_done=*/true);
  if (e != cudaSuccess) return e;
  // 5. ranges (the pointer pair lives in the header's spare words)
  uint2 *ranges = region<uint2>(p, ws, R_RANGES);
  e = cudaMemsetAsync(ranges, 0, p->bytes[R_RANGES], s);
  if (e != cudaSuccess) return e;
  k_ranges<<<g_stream_blocks, 256, 0, s>>>(t.keys[0], t.keys[1], &hdr->sel_pair, &hdr->n_pairs,
                                         p->max_pairs, ranges);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Allocation-free variant of the pair sort (no counterpart in the paper).
//
// Some callers cannot allocate device memory at all: code running inside a
// memory pool that must not grow, plug-ins whose host forbids cudaMalloc
// after start-up, or real-time paths where an allocation could block.  For
// them gs_sort_pairs_static sorts caller-provided buffers using a fixed
// scratch array that lives in this file as a static device variable, sized
// for at most GS_STATIC_SORT_MAX_PAIRS pairs.  Every GPU that loads the
// library holds that array (about 9 MB) until the process exits.
// --------------------------------------------------------------------------
namespace {

constexpr long long kStaticMax = GS_STATIC_SORT_MAX_PAIRS;
constexpr long long kStaticParts = (kStaticMax + kSortPart - 1) / kSortPart;

struct StaticHdr {
  unsigned long long count;
  uint32_t hist[4][256];
  uint32_t skip[4];
  uint32_t tickets[4];
  uint32_t sel;
  uint32_t status;
};

constexpr size_t kStaticHdrBytes = (sizeof(StaticHdr) + 255) & ~size_t(255);
constexpr size_t kStaticTmpBytes = 2 * sizeof(uint32_t) * (size_t)kStaticMax;   // keys + values
constexpr size_t kStaticLbBytes = 2 * 256 * sizeof(unsigned long long) * (size_t)kStaticParts;
constexpr size_t kStaticBytes = kStaticHdrBytes + kStaticTmpBytes + kStaticLbBytes;

// The scratch itself.  Host code must not take this symbol's address
// directly (that would be a host-side stand-in); it asks the runtime for the
// device address once per device.
static __device__ __align__(256) unsigned char g_sort_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned char *g_static_ptr[kMaxDevices] = {};

__global__ void k_static_set_count(StaticHdr *h, unsigned long long n) {
  h->count = n;
  h->status = 0u;
}

}  // namespace

}  // namespace gs

extern "C" gs_status gs_sort_pairs_static(const uint32_t *keys_in, const uint32_t *vals_in,
                                           int64_t n, int32_t key_bits, uint32_t *keys_out,
                                           uint32_t *vals_out, cudaStream_t stream) {
  using namespace gs;
  if (n < 0 || n > kStaticMax || key_bits < 1 || key_bits > 32) return GS_ERR_INVALID_ARG;
  if (n > 0 && (!keys_in || !vals_in || !keys_out || !vals_out)) return GS_ERR_INVALID_ARG;
  // the buffers must not overlap (the first pass reads the input while
  // writing the output)
  auto overlap = [n](const void *a, const void *b) {
    const char *x = static_cast<const char *>(a), *y = static_cast<const char *>(b);
    return x < y + 4 * n && y < x + 4 * n;
  };
  if (n > 0 && (overlap(keys_in, keys_out) || overlap(vals_in, vals_out) ||
                overlap(keys_in, vals_out) || overlap(vals_in, keys_out) ||
                overlap(keys_out, vals_out)))
    return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GS_ERR_CUDA;
  unsigned char *base;
  {
    // one-time set-up per device, with that device current
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_sort_scratch) != cudaSuccess || !ptr) return GS_ERR_CUDA;
      g_static_ptr[dev] = static_cast<unsigned char *>(ptr);
    }
    base = g_static_ptr[dev];
  }
  StaticHdr *h = reinterpret_cast<StaticHdr *>(base);
  uint32_t *tmp_k = reinterpret_cast<uint32_t *>(base + kStaticHdrBytes);
  uint32_t *tmp_v = tmp_k + kStaticMax;
  unsigned long long *lb = reinterpret_cast<unsigned long long *>(base + kStaticHdrBytes + kStaticTmpBytes);
  // the array keeps the previous call's contents: clear what must start at 0
  if (cudaMemsetAsync(h, 0, sizeof(StaticHdr), stream) != cudaSuccess) return GS_ERR_CUDA;
  k_static_set_count<<<1, 1, 0, stream>>>(h, (unsigned long long)n);
  SortArgs a = {};
  a.passes = (key_bits + 7) / 8;
  a.digit_bits = (key_bits + a.passes - 1) / a.passes;
  a.first_keys = keys_in;
  a.first_vals = vals_in;
  // every pass runs, so pass p writes buffer (p + 1) & 1: put the caller's
  // output where the last pass writes
  const int last = a.passes & 1;
  a.keys[last] = keys_out;
  a.vals[last] = vals_out;
  a.keys[last ^ 1] = tmp_k;
  a.vals[last ^ 1] = tmp_v;
  a.count = &h->count;
  a.capacity = kStaticMax;
  a.sel = &h->sel;
  a.hist = &h->hist[0][0];
  a.skip = &h->skip[0];
  a.tickets = &h->tickets[0];
  a.lb = lb;
  a.max_parts = kStaticParts;
  a.no_skip = 1;
  a.status = &h->status;
  return run_sort(a, stream) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
