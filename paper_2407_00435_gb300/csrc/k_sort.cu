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
// Each radix pass is reduce-then-scan over a fixed grid of G blocks, block b
// owning one contiguous range of 4096-key partitions:
//   upsweep    per-block digit counts of the range            (reads keys)
//   scan       per digit, exclusive scan over the G blocks, plus the
//              digit's global start                            (G x 256)
//   downsweep  the block walks its partitions in order with a running
//              per-digit carry (next partition prefetched by bulk copy):
//              rank digits inside each warp (peer lanes by one ballot per
//              digit bit), stage the partition in digit order in shared
//              memory, write runs of equal digits contiguously.
// No block waits for another (no look-back chain, no spin).  The global
// histograms of every pass come from one read of the keys (or from the
// emit); a pass whose digit is the same for all keys is skipped on the
// device.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <mutex>

#include "gs_internal.cuh"
#include "support.cuh"
#include "tma.cuh"

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
  uint32_t *bsum;                    // [G][256] per-block digit counts -> bases
  int blocks;                        // G, the grid of upsweep and downsweep
  int passes;
  int digit_bits;                    // bits per pass (<= 8)
  int key_bits;                      // significant bits of the keys (0: passes x digit_bits);
                                     //   the last pass ranks only the bits left
  int no_skip;                       // run every pass (fixed buffer parity)
  const uint32_t *key_range;         // cooperative sort: (largest kept key, complement of the
                                     //   smallest), or null (see k_sort_coop)
  int drop_max;                      // cooperative sort: the first pass drops keys equal
                                     //   to 0xffffffff (the result holds the others only)
  uint2 *ranges;                     // cooperative sort: [start, end) of each key value in
  long long n_ranges;                //   the result (keys < n_ranges; zeroed by the caller)
  int extra_zeroed;                  // cooperative sort: the caller cleared the barrier word
                                     //   and the first parity of sums (coop_extra)
  uint32_t *status;
  int sub;                           // upsweep sub-ranges per block, 1..kSortSub (0: kSortSub)
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

// Partition ranges: downsweep block b of G owns partitions [b q, (b + 1) q),
// q = ceil(parts / G).  The upsweep splits each block's key range into
// `sub` equal pieces (it only counts, so any split is fine); row s of the
// block table belongs to piece s % sub of block s / sub.
__device__ __forceinline__ void block_parts(uint32_t n, int G, int b, long long &p0, long long &p1) {
  const long long nparts = ((long long)n + kSortPart - 1) / kSortPart;
  const long long q = (nparts + G - 1) / G;
  p0 = (long long)b * q < nparts ? (long long)b * q : nparts;
  p1 = p0 + q < nparts ? p0 + q : nparts;
}

__device__ __forceinline__ void sub_keys(uint32_t n, int G, int sub, long long s, long long &k0,
                                         long long &k1) {
  long long p0, p1;
  block_parts(n, G, (int)(s / sub), p0, p1);
  const long long b0 = p0 * kSortPart;
  const long long b1 = p1 * kSortPart < (long long)n ? p1 * kSortPart : (long long)n;
  const long long len = b1 > b0 ? b1 - b0 : 0;
  const long long j = s % sub;
  k0 = b0 + len * j / sub;
  k1 = b0 + len * (j + 1) / sub;
}

// Input buffers of pass `pass`: the first executed pass reads the caller's
// arrays, later ones the ping-pong buffer the previous executed pass wrote.
__device__ __forceinline__ int passes_before(const SortArgs &a, int pass) {
  int before = 0;
  for (int p = 0; p < pass; ++p) before += a.skip[p] ? 0 : 1;
  return before;
}

// Adds digit d of the valid lanes to a shared histogram; a warp whose
// valid lanes share one digit (common for the high bytes of depth keys)
// adds once.
__device__ __forceinline__ void warp_count(uint32_t *h, bool valid, uint32_t d, int lane) {
  const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
  if (!vmask) return;
  const uint32_t d0 = __shfl_sync(0xffffffffu, d, __ffs(vmask) - 1);
  if (__all_sync(0xffffffffu, !valid || d == d0)) {
    if (lane == __ffs(vmask) - 1) atomicAdd(&h[d0], (uint32_t)__popc(vmask));
  } else if (valid) {
    atomicAdd(&h[d], 1u);
  }
}

// ---- histograms of every pass in one read of the keys ---------------------
constexpr int kHistUnroll = 8;

__global__ void __launch_bounds__(256) k_hist(SortArgs a) {
  __shared__ uint32_t sh[4][256];
  const uint32_t n = sort_n(a);
  for (int q = threadIdx.x; q < 4 * 256; q += blockDim.x) (&sh[0][0])[q] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x * kHistUnroll;
  const uint32_t dmask = (1u << a.digit_bits) - 1u;
  // warp-uniform trip count so that the warp votes see the full warp
  for (long long base = (long long)blockIdx.x * blockDim.x * kHistUnroll; base < (long long)n;
       base += stride) {
    uint32_t key[kHistUnroll];
#pragma unroll
    for (int u = 0; u < kHistUnroll; ++u) {
      const long long idx = base + u * blockDim.x + threadIdx.x;
      key[u] = idx < (long long)n ? a.first_keys[idx] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kHistUnroll; ++u) {
      const bool valid = base + u * blockDim.x + threadIdx.x < (long long)n;
      for (int p = 0; p < a.passes; ++p)
        warp_count(sh[p], valid, (key[u] >> (a.digit_bits * p)) & dmask, lane);
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < a.passes * 256; q += blockDim.x) {
    uint32_t c = (&sh[0][0])[q];
    if (c) atomicAdd(&a.hist[q], c);
  }
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

// ---- upsweep: digit counts of each sub-range (sub x G blocks) ----------------
constexpr int kUpUnroll = 8;

__global__ void __launch_bounds__(kSortThreads) k_upsweep(SortArgs a, int pass) {
  __shared__ uint32_t s_h[kSortThreads / 32][256];
  if (a.skip[pass]) return;
  const uint32_t n = sort_n(a);
  const int before = passes_before(a, pass);
  const uint32_t *kin = before == 0 ? a.first_keys : ((before & 1) ? a.keys[1] : a.keys[0]);
  const int shift = a.digit_bits * pass;
  const uint32_t dmask = (1u << a.digit_bits) - 1u;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int q = tid; q < (kSortThreads / 32) * 256; q += kSortThreads) (&s_h[0][0])[q] = 0u;
  __syncthreads();
  long long k0, k1;
  sub_keys(n, a.blocks, a.sub, blockIdx.x, k0, k1);
  constexpr int kStep = kSortThreads * kUpUnroll;
  for (long long base = k0; base < k1; base += kStep) {
    uint32_t key[kUpUnroll];
#pragma unroll
    for (int u = 0; u < kUpUnroll; ++u) {
      const long long idx = base + u * kSortThreads + tid;
      key[u] = idx < k1 ? kin[idx] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kUpUnroll; ++u) {
      const long long idx = base + u * kSortThreads + tid;
      warp_count(s_h[warp], idx < k1, (key[u] >> shift) & dmask, lane);
    }
  }
  __syncthreads();
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < kSortThreads / 32; ++w) tot += s_h[w][tid];
  a.bsum[(long long)blockIdx.x * 256 + tid] = tot;
}

// ---- scan: bsum[s][d] <- global start of digit d + its count in
// sub-ranges < s.  One block per 8 digits (one 32-byte sector of a table
// row); thread (slice, digit) owns a run of rows of its digit, so each load
// instruction of a warp reads whole sectors of 4 rows.  Up to kScanRegRows
// rows per thread stay in registers between the two phases (one read of the
// table); longer runs are read twice, kScanChunk at a time.
constexpr int kScanThreads = 1024;
constexpr int kScanDigits = 8;
constexpr int kScanSlices = kScanThreads / kScanDigits;
constexpr int kScanChunk = 16;
constexpr int kScanRegRows = 32;

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(SortArgs a, int pass) {
  __shared__ uint32_t s_p[kScanDigits][kScanSlices + 1];
  if (a.skip[pass]) return;
  const int R = a.sub * a.blocks;
  const int dl = threadIdx.x & (kScanDigits - 1), sl = threadIdx.x / kScanDigits;
  const int d = blockIdx.x * kScanDigits + dl;
  const int rows = (R + kScanSlices - 1) / kScanSlices;
  const int r0 = sl * rows < R ? sl * rows : R;
  const int r1 = r0 + rows < R ? r0 + rows : R;
  const bool in_regs = rows <= kScanRegRows;
  uint32_t v[kScanRegRows];
  uint32_t sum = 0;
  if (in_regs) {
#pragma unroll
    for (int i = 0; i < kScanRegRows; ++i)
      v[i] = r0 + i < r1 ? a.bsum[(long long)(r0 + i) * 256 + d] : 0u;
#pragma unroll
    for (int i = 0; i < kScanRegRows; ++i) sum += v[i];
  } else {
    for (int c = r0; c < r1; c += kScanChunk) {
      uint32_t w[kScanChunk];
#pragma unroll
      for (int i = 0; i < kScanChunk; ++i) w[i] = c + i < r1 ? a.bsum[(long long)(c + i) * 256 + d] : 0u;
#pragma unroll
      for (int i = 0; i < kScanChunk; ++i) sum += w[i];
    }
  }
  s_p[dl][sl] = sum;
  __syncthreads();
  // warp w < 8: exclusive scan of digit w's slice sums (4 slices per lane)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  static_assert(kScanSlices == 4 * 32, "4 slices per lane");
  if (warp < kScanDigits) {
    uint32_t x[4], loc = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      x[i] = s_p[warp][4 * lane + i];
      loc += x[i];
    }
    uint32_t incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t run = a.hist[pass * 256 + blockIdx.x * kScanDigits + warp] + incl - loc;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      s_p[warp][4 * lane + i] = run;
      run += x[i];
    }
  }
  __syncthreads();
  uint32_t run = s_p[dl][sl];
  if (in_regs) {
#pragma unroll
    for (int i = 0; i < kScanRegRows; ++i) {
      if (r0 + i < r1) a.bsum[(long long)(r0 + i) * 256 + d] = run;
      run += v[i];
    }
  } else {
    for (int c = r0; c < r1; c += kScanChunk) {
      uint32_t w[kScanChunk];
#pragma unroll
      for (int i = 0; i < kScanChunk; ++i) w[i] = c + i < r1 ? a.bsum[(long long)(c + i) * 256 + d] : 0u;
#pragma unroll
      for (int i = 0; i < kScanChunk; ++i) {
        if (c + i < r1) a.bsum[(long long)(c + i) * 256 + d] = run;
        run += w[i];
      }
    }
  }
}

// ---- downsweep: rank, stage in digit order, scatter -----------------------
// Each block walks its partitions in order.  While one partition is ranked
// and scattered, the next one's keys and values are already on their way
// into the other half of a double buffer by two bulk copies (thread 0
// issues them; an mbarrier per half counts the bytes in).  Partitions that
// are not full, or inputs that are not 16-byte aligned, are read with plain
// loads instead.
template <int NT, int NBK = 256>     // NBK digit values (256, 512 or 1024): digits of up to
                                     //   log2(NBK) bits
struct DownSmemT {
  static_assert(NT >= NBK, "one thread per digit value");
  uint32_t in_k[2][kSortPart];
  uint32_t in_v[2][kSortPart];
  uint32_t key[kSortPart];            // staging in digit order
  uint32_t val[kSortPart];
  uint16_t wh[NT / 32][NBK];          // per-warp digit counts, then offsets
  uint32_t base[NBK], carry[NBK], dstart[NBK];
  uint32_t wsum[NBK / 32];            // the digit threads' warp sums
  uint64_t bar[2];
};
using DownSmem = DownSmemT<kDownThreads>;

// Bookkeeping of the two halves of the downsweep's double buffer (copies
// issued and consumed); block-uniform, kept across the passes of one launch.
struct DownBufs {
  uint32_t issued0, issued1, used0, used1;
};

// Ranks the ITEMS keys of each lane of the warp (item k of lane l is key
// k * 32 + l of the warp's slice): rank[k] = the key's position among the
// warp's keys of the same digit so far; sm.wh[warp][d] counts them.  RB
// ballots (the digit width rounded up); ALLV: every key is kept.
template <int RB, bool ALLV, int NT, int NBK, int ITEMS>
__device__ __forceinline__ void rank_items(const uint32_t (&key)[ITEMS], uint32_t (&rank)[ITEMS],
                                           DownSmemT<NT, NBK> &sm, int warp, int lane,
                                           uint32_t ltmask, int shift, uint32_t dmask, int lbase,
                                           int rem, bool drop) {
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const bool valid = ALLV || ((lbase + k * 32 + lane < rem) && !(drop && key[k] == 0xffffffffu));
    const uint32_t d = (key[k] >> shift) & dmask;
    uint32_t peers = ALLV ? 0xffffffffu : __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int bit = 0; bit < RB; ++bit) {
      const bool set = ((d >> bit) & 1u) != 0u;
      const uint32_t bb = __ballot_sync(0xffffffffu, set);
      peers &= set ? bb : ~bb;
    }
    const uint32_t before_w = valid ? (uint32_t)sm.wh[warp][d] : 0u;
    rank[k] = before_w + __popc(peers & ltmask);
    __syncwarp();
    if (valid && (__ffs(peers) - 1) == lane) sm.wh[warp][d] = (uint16_t)(before_w + __popc(peers));
    __syncwarp();
  }
}

// Walks partitions [p0, p1) of pass `pass` in order, sm.carry[d] holding
// the output position of the next key of digit d.  `before` = executed
// passes before this one (selects the buffers).  `drop`: keys equal to
// 0xffffffff are left out (not ranked, staged or written; the bases count
// only the others).  `dbits`: digit width of the pass; `kmin`: subtracted
// from every kept key as it is read (0: keys as they are); `rbits`: the
// digit's significant bits in this pass (fewer in a last pass), the ballots
// the ranking takes.  Returns false if
// a bounded wait gave up (status set, copies in flight drained).
template <int NT, int NBK = 256>
__device__ __forceinline__ bool downsweep_range(const SortArgs &a, int pass, int before,
                                                DownSmemT<NT, NBK> &sm, DownBufs &db,
                                                long long p0, long long p1, uint32_t n,
                                                bool drop, int dbits, uint32_t kmin, int rbits) {
  constexpr int NW = NT / 32;
  constexpr int ITEMS = kSortPart / NT;
  constexpr int NBITS = NBK == 1024 ? 10 : (NBK == 512 ? 9 : 8);
  constexpr int NDW = NBK / 32;   // warps of the digit threads
  const bool odd = (before & 1) != 0;   // (no dynamic indexing of the parameter arrays)
  const uint32_t *kin = before == 0 ? a.first_keys : (odd ? a.keys[1] : a.keys[0]);
  const uint32_t *vin = before == 0 ? a.first_vals : (odd ? a.vals[1] : a.vals[0]);
  uint32_t *kout = odd ? a.keys[0] : a.keys[1];
  uint32_t *vout = odd ? a.vals[0] : a.vals[1];
  const bool iota = vin == nullptr;
  const int shift = dbits * pass;
  const uint32_t dmask = (1u << rbits) - 1u;   // (keys have no bits above: nothing is lost)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t ltmask = lanemask_lt();
  const bool aligned = ((uintptr_t)kin & 15u) == 0 && (iota || ((uintptr_t)vin & 15u) == 0);
  const long long full = (long long)n / kSortPart;   // partitions [0, full) hold 4096 keys
  constexpr uint32_t kBytes = kSortPart * sizeof(uint32_t);
  auto issue = [&](long long part, int h) {
    if (tid == 0) {
      fence_proxy_async_smem();
      mbar_expect_tx(&sm.bar[h], iota ? kBytes : 2 * kBytes);
      bulk_g2s(sm.in_k[h], kin + part * kSortPart, kBytes, &sm.bar[h]);
      if (!iota) bulk_g2s(sm.in_v[h], vin + part * kSortPart, kBytes, &sm.bar[h]);
    }
    if (h) ++db.issued1; else ++db.issued0;
  };
  // half 0 is refilled first in every range (the previous range consumed
  // every copy it issued)
  if (aligned && p0 < p1 && p0 < full) issue(p0, 0);
  int h = 0;
  for (long long part = p0; part < p1; ++part, h ^= 1) {
    const bool bulk = aligned && part < full;
    // the other half was last read before the barrier ending the previous
    // partition: refill it with the next partition
    if (part + 1 < p1 && aligned && part + 1 < full) issue(part + 1, h ^ 1);
    for (int q = tid; q < NW * NBK / 2; q += NT)
      reinterpret_cast<uint32_t *>(&sm.wh[0][0])[q] = 0u;
    const long long pbase = part * kSortPart;
    // keys of this partition: local indices [0, rem)
    const int rem = (int)min((long long)kSortPart, (long long)n - pbase);
    const int lbase = warp * (32 * ITEMS);
    uint32_t key[ITEMS], rank[ITEMS];
    if (bulk) {
      const uint32_t u = h ? db.used1 : db.used0;
      const bool landed = mbar_wait_bounded(&sm.bar[h], u & 1u);
      if (h) ++db.used1; else ++db.used0;
      if (__syncthreads_or(!landed)) {
        // give up: record it, let the copies in flight land, leave
        if (tid == 0) set_status(a.status, GS_ERR_TIMEOUT);
        if (db.issued0 > db.used0) mbar_wait_bounded(&sm.bar[0], db.used0 & 1u);
        if (db.issued1 > db.used1) mbar_wait_bounded(&sm.bar[1], db.used1 & 1u);
        return false;
      }
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) key[k] = sm.in_k[h][lbase + k * 32 + lane];
    } else {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const int li = lbase + k * 32 + lane;
        key[k] = li < rem ? __ldcg(&kin[pbase + li]) : 0u;
      }
    }
    if (kmin) {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) key[k] = key[k] == 0xffffffffu ? key[k] : key[k] - kmin;
    }
    __syncthreads();
    // warp-level stable ranking (original order = (k, lane)); the lanes
    // holding the same digit are found with one ballot per digit bit (bits
    // above the digit width are zero in every lane: their ballots are 0 and
    // leave the mask as it is).  Specialised for digits of at most 7 bits
    // (one ballot less) and for partitions whose keys are all kept.
    const bool allv = rem == kSortPart && !drop;
#define GS_RANK(R)                                                                              \
  do {                                                                                          \
    if (allv) rank_items<R, true, NT, NBK>(key, rank, sm, warp, lane, ltmask, shift, dmask,     \
                                           lbase, rem, drop);                                   \
    else rank_items<R, false, NT, NBK>(key, rank, sm, warp, lane, ltmask, shift, dmask, lbase,  \
                                       rem, drop);                                              \
  } while (0)
    if (NBK == 256) {
      if (rbits <= 6) GS_RANK(6);
      else if (rbits == 7) GS_RANK(7);
      else GS_RANK(8);
    } else if (NBK == 512) {
      if (rbits <= 8) GS_RANK(8);
      else GS_RANK(9);
    } else {
      if (rbits <= 9) GS_RANK(9);
      else GS_RANK(10);
    }
#undef GS_RANK
    __syncthreads();
    // per digit (threads 0..255): warp offsets inside the partition, the
    // running base, and the digit's start inside the partition
    uint32_t tot = 0, incl = 0;
    if (tid < NBK) {
      const int d = tid;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t c = sm.wh[w][d];
        sm.wh[w][d] = (uint16_t)tot;
        tot += c;
      }
      sm.base[d] = sm.carry[d];
      sm.carry[d] += tot;
      incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (lane == 31) sm.wsum[warp] = incl;
    }
    __syncthreads();
    if (tid < NBK) {
      uint32_t wofs = 0;
#pragma unroll
      for (int w = 0; w < NDW; ++w) wofs += w < warp ? sm.wsum[w] : 0u;
      sm.dstart[tid] = wofs + incl - tot;
    }
    // keys staged: every key of the partition, or the kept ones
    uint32_t pcount = (uint32_t)rem;
    if (drop) {
      pcount = 0;
#pragma unroll
      for (int w = 0; w < NDW; ++w) pcount += sm.wsum[w];
    }
    __syncthreads();
    // stage the partition in digit order, then write runs of equal digits
    // to consecutive global addresses
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const int li = lbase + k * 32 + lane;
      if (li < rem && !(drop && key[k] == 0xffffffffu)) {
        const uint32_t d = (key[k] >> shift) & dmask;
        const uint32_t lp = sm.dstart[d] + (uint32_t)sm.wh[warp][d] + rank[k];
        sm.key[lp] = key[k];
        sm.val[lp] = iota ? (uint32_t)(pbase + li) : (bulk ? sm.in_v[h][li] : __ldcg(&vin[pbase + li]));
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint32_t lp = (uint32_t)(k * NT + tid);
      if (lp < pcount) {
        const uint32_t kk = sm.key[lp];
        const uint32_t d = (kk >> shift) & dmask;
        const uint32_t dst = sm.base[d] + (lp - sm.dstart[d]);
        if (dst < n) {
          kout[dst] = kk;
          vout[dst] = sm.val[lp];
        }
      }
    }
    __syncthreads();
  }
  return true;
}

__global__ void __launch_bounds__(kDownThreads, 2) k_downsweep(SortArgs a, int pass) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  DownSmem &sm = *reinterpret_cast<DownSmem *>(dyn_smem);
  if (a.skip[pass]) return;
  const uint32_t n = sort_n(a);
  long long p0, p1;
  block_parts(n, a.blocks, blockIdx.x, p0, p1);
  if (p0 >= p1) return;
  const int tid = threadIdx.x;
  if (tid < 256) sm.carry[tid] = a.bsum[(long long)blockIdx.x * a.sub * 256 + tid];
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  DownBufs db = {0u, 0u, 0u, 0u};
  downsweep_range<kDownThreads>(a, pass, passes_before(a, pass), sm, db, p0, p1, n, false,
                                a.digit_bits, 0u, a.digit_bits);
}

// ---- the whole sort in one cooperative launch -------------------------------
// Every pass of the sort in one launch of G co-resident blocks (cooperative
// launch), block b owning the partitions block_parts(n, G, b):
//   count    block b's digit counts -> row b of a table (double-buffered by
//            pass parity)
//   barrier  every row written
//   bases    each block reads the table's columns: the digit totals (digit
//            starts by an exclusive scan) and the counts of the blocks
//            before it -> its running per-digit output positions; a digit
//            that every key shares skips the pass (all blocks agree)
//   scatter  downsweep_range over the block's partitions
//   barrier  the pass's output complete before the next pass reads it
// The barriers count arrivals on one global word that only grows (zeroed
// before the launch): the e-th barrier is passed once it reaches e G.  They
// replace the 3 launches per pass (and the fixed latency of each) of the
// multi-kernel sort.
//
// So that no block reads the whole table, the count also adds each block's
// digit counts, by atomics, to the digit totals and to the sums of its group
// of kCoopGroup blocks: a block's bases are then the totals, the group sums
// of the groups before it and the rows of its own group before it (at most
// 1 + G / kCoopGroup + kCoopGroup - 1 rows instead of G).
//
// Layout after the two G x 256 tables in a.bsum (uint32 words): the barrier
// word (64 words reserved), then per pass parity kCoopSumRows rows of 256:
// row 0 the totals, row 1 + g the sums of group g.  The barrier word and
// parity 0 are zeroed before the launch; parity q ^ 1 is zeroed by block 0
// during a pass of parity q (after its first barrier: every block has left
// the previous pass, and the next pass adds only after this pass's second
// barrier).
struct CoopBar {
  unsigned int count;
  unsigned int spare;
};
constexpr int kCoopGroup = 16;                      // blocks per group of the bases
constexpr int kCoopMaxGroups = 64;                  // grids of up to 1024 blocks
constexpr int kCoopSumRows = 1 + kCoopMaxGroups;    // totals + group sums, per parity
// rows of 256 words a cooperative sort of G blocks and NBK digit values needs
// in a.bsum: two G x NBK tables, the barrier word, two parities of sums
__host__ __device__ constexpr long long coop_table_rows(int G, int NBK = 256) {
  return (2LL * G * NBK + 64 + 2LL * kCoopSumRows * NBK + 255) / 256;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch, bounded: false (status set)
// if the other blocks did not all arrive within the limit.  `epoch`: the
// barriers this block passed (thread 0's copy).  One atomic per block and
// no second word: the last block to arrive releases the others by its add.
__device__ __forceinline__ bool grid_barrier(CoopBar *bar, unsigned int &epoch, uint32_t *status,
                                             int *s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    const unsigned int target = epoch * gridDim.x;
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar->count, 1u) + 1u;
    bool ok = true;
    if ((int)(arrived - target) < 0) {
      // (blocks already past this barrier may have added for the next one)
      int it = 0;
      while ((int)(ld_acquire_u32(&bar->count) - target) < 0) {
        if (++it > kSpinLimit) {
          ok = false;
          set_status(status, GS_ERR_TIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    // the bulk copies this thread issues next read, through the async
    // proxy, what other blocks wrote through the generic proxy
    asm volatile("fence.proxy.async.global;" ::: "memory");
    *s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  return *s_ok != 0;
}

constexpr int kCountUnroll = 8;

// NT threads per block: launched with one block per SM (the depth sort:
// half of each SM stays free for the pair count, which runs beside it and
// fills the sort's barrier waits) or two (the pair sort: a block's
// partitions overlap the other block's).
//
// With a.key_range (NBK = 512), the keys are the visible depth keys: the
// first pass subtracts the smallest kept key from every kept key, and the
// digit width and pass count follow from the span of the kept keys (9-bit
// digits: a span of 2^27 sorts in 3 passes instead of 4), the same in every
// block.
template <int NT, int NBK>
__global__ void __launch_bounds__(NT, 1024 / NT) k_sort_coop(SortArgs a) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  DownSmemT<NT, NBK> &sm = *reinterpret_cast<DownSmemT<NT, NBK> *>(dyn_smem);
  constexpr int kCoopThreads = NT;
  constexpr int NDW = NBK / 32;   // warps of the digit threads
  __shared__ uint32_t s_cnt[NBK];
  __shared__ uint32_t s_wsum[NDW];
  __shared__ int s_ok, s_skip;
  // keys of the current pass (after a dropping first pass: the kept ones)
  uint32_t n = sort_n(a);
  const int G = gridDim.x, b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31;
  int dbits = a.digit_bits, npasses = a.passes;
  int kbits = a.key_bits > 0 ? a.key_bits : a.digit_bits * a.passes;
  uint32_t kmin = 0;
  if (NBK == 512 && a.key_range) {
    // key_range = (largest kept key, complement of the smallest)
    const uint32_t kmax = a.key_range[0], lo = ~a.key_range[1];
    const uint32_t span = kmax >= lo ? kmax - lo : 0u;
    const int bits = span ? 32 - __clz(span) : 1;
    dbits = 9;
    npasses = (bits + 8) / 9;
    kmin = lo;
    kbits = bits;
  }
  const bool force_first = a.first_vals == nullptr;
  uint32_t *extra = a.bsum + (size_t)2 * G * NBK;
  CoopBar *bar = reinterpret_cast<CoopBar *>(extra);
  uint32_t *sums_base = extra + 64;
  const int grp = b / kCoopGroup;
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_fence_init();
  }
  DownBufs db = {0u, 0u, 0u, 0u};
  int executed = 0;
  unsigned int epoch = 0;
  for (int pass = 0; pass < npasses; ++pass) {
    const bool odd = (executed & 1) != 0;
    const uint32_t *kin = executed == 0 ? a.first_keys : (odd ? a.keys[1] : a.keys[0]);
    const int shift = dbits * pass;
    const bool drop = a.drop_max != 0 && pass == 0;
    const uint32_t ksub = pass == 0 ? kmin : 0u;   // keys are relative once written
    // this pass's significant digit bits (the last pass may have fewer)
    const int rbits = min(dbits, max(1, kbits - shift));
    const uint32_t pmask = (1u << rbits) - 1u;
    long long p0, p1;
    block_parts(n, G, b, p0, p1);
    const long long k0 = p0 * kSortPart;
    const long long k1 = p1 * kSortPart < (long long)n ? p1 * kSortPart : (long long)n;
    uint32_t *table = a.bsum + (size_t)(pass & 1) * (size_t)G * NBK;
    uint32_t *sums = sums_base + (size_t)(pass & 1) * kCoopSumRows * NBK;
    // count
    if (tid < NBK) s_cnt[tid] = 0u;
    __syncthreads();
    const int warp = tid >> 5;
    for (long long base = k0 + (long long)warp * 32 * kCountUnroll; base < k1;
         base += (long long)kCoopThreads * kCountUnroll) {
      uint32_t key[kCountUnroll];
#pragma unroll
      for (int u = 0; u < kCountUnroll; ++u) {
        const long long idx = base + u * 32 + lane;
        key[u] = idx < k1 ? __ldcg(&kin[idx]) : 0u;
      }
#pragma unroll
      for (int u = 0; u < kCountUnroll; ++u)
        warp_count(s_cnt, base + u * 32 + lane < k1 && !(drop && key[u] == 0xffffffffu),
                   ((key[u] - ksub) >> shift) & pmask, lane);
    }
    __syncthreads();
    if (tid < NBK) {
      const uint32_t c = s_cnt[tid];
      table[(size_t)b * NBK + tid] = c;
      if (c) {
        atomicAdd(&sums[tid], c);
        atomicAdd(&sums[(size_t)(1 + grp) * NBK + tid], c);
      }
    }
    if (!grid_barrier(bar, epoch, a.status, &s_ok)) return;
    if (b == 0) {
      // the other parity's sums, for the next pass
      uint32_t *nxt = sums_base + (size_t)((pass + 1) & 1) * kCoopSumRows * NBK;
      for (int q = tid; q < kCoopSumRows * NBK / 4; q += kCoopThreads)
        reinterpret_cast<uint4 *>(nxt)[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    // bases: digit d's total over all blocks (row 0 of the sums) and its
    // count in blocks < b: the sums of groups < grp and the table rows of
    // blocks grp * kCoopGroup .. b - 1.  Thread t adds 4 digits (16-byte
    // loads) of rows t / (NBK / 4), + NG, ... of that list; the NG row
    // groups' partial sums meet in the staging buffers (free between the
    // passes' scatters)
    {
      constexpr int NQ = NBK / 4;   // 16-byte words per row
      constexpr int NG = kCoopThreads / NQ;
      static_assert(NG * NBK <= kSortPart, "partials fit the staging buffer");
      const int dg = tid & (NQ - 1), rg = tid / NQ;
      const uint4 *tab4 = reinterpret_cast<const uint4 *>(table);
      const uint4 *sum4 = reinterpret_cast<const uint4 *>(sums);
      const int b0 = grp * kCoopGroup;
      const int nrows = grp + (b - b0);   // group sums, then own group's earlier rows
      uint4 p4 = make_uint4(0u, 0u, 0u, 0u);
      for (int r0 = rg; r0 < nrows; r0 += NG * 4) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = r0 + u * NG;
          v[u] = r >= nrows ? make_uint4(0u, 0u, 0u, 0u)
                            : (r < grp ? __ldcg(&sum4[(size_t)(1 + r) * NQ + dg])
                                       : __ldcg(&tab4[(size_t)(b0 + r - grp) * NQ + dg]));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          p4.x += v[u].x; p4.y += v[u].y; p4.z += v[u].z; p4.w += v[u].w;
        }
      }
      reinterpret_cast<uint4 *>(sm.val)[rg * NQ + dg] = p4;
      if (rg == 0) reinterpret_cast<uint4 *>(sm.key)[dg] = __ldcg(&sum4[dg]);
    }
    if (tid == 0) s_skip = 0;
    __syncthreads();
    uint32_t tot = 0, incl = 0, pre = 0;
    if (tid < NBK) {
      tot = sm.key[tid];
#pragma unroll
      for (int q = 0; q < kCoopThreads / (NBK / 4); ++q) pre += sm.val[q * NBK + tid];
      if (tot == n) s_skip = 1;   // one digit holds every key
      incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (lane == 31) s_wsum[tid >> 5] = incl;
    }
    __syncthreads();
    // a dropping pass always runs (it changes the key set); the keys it keeps
    // are the table's total (the same in every block)
    uint32_t n_out = n;
    if (drop) {
      n_out = 0;
#pragma unroll
      for (int w = 0; w < NDW; ++w) n_out += s_wsum[w];
    }
    const bool skip = (s_skip || n == 0) && !drop &&
                      !(force_first && executed == 0 && pass == npasses - 1) && !a.no_skip;
    if (skip) {
      // nothing written; the barrier keeps the sums' zeroing ordered
      if (!grid_barrier(bar, epoch, a.status, &s_ok)) return;
      continue;
    }
    if (tid < NBK) {
      uint32_t wofs = 0;
#pragma unroll
      for (int w = 0; w < NDW; ++w) wofs += w < (tid >> 5) ? s_wsum[w] : 0u;
      sm.carry[tid] = wofs + incl - tot + pre;
    }
    __syncthreads();
    if (p0 < p1 && !downsweep_range<NT, NBK>(a, pass, executed, sm, db, p0, p1, n, drop, dbits,
                                             ksub, rbits)) {
      // leave the grid barrier to time out in the other blocks
      return;
    }
    ++executed;
    n = n_out;
    if (!grid_barrier(bar, epoch, a.status, &s_ok)) return;
  }
  if (b == 0 && tid == 0) *a.sel = (uint32_t)(executed & 1);
  if (a.ranges) {
    // per key value (tile) its range in the sorted keys: block b marks the
    // starts and ends that fall in its own partitions
    const uint32_t *key = (executed & 1) ? a.keys[1] : a.keys[0];
    long long p0, p1;
    block_parts(n, G, b, p0, p1);
    const long long k0 = p0 * kSortPart;
    const long long k1 = p1 * kSortPart < (long long)n ? p1 * kSortPart : (long long)n;
    for (long long q = k0 + tid; q < k1; q += kCoopThreads) {
      const uint32_t k = __ldcg(&key[q]);
      const uint32_t kp = q > 0 ? __ldcg(&key[q - 1]) : ~0u;
      const uint32_t kn = q + 1 < (long long)n ? __ldcg(&key[q + 1]) : ~0u;
      if ((long long)k >= a.n_ranges) {   // never written by a consistent emit
        set_status(a.status, GS_ERR_CUDA);
        continue;
      }
      if (q == 0 || kp != k) a.ranges[k].x = (uint32_t)q;
      if (q == (long long)n - 1 || kn != k) a.ranges[k].y = (uint32_t)(q + 1);
    }
  }
}

static int g_sort_blocks = 0;
static int g_stream_blocks = 0;   // grid of the streaming kernels (emit, offsets, ranges, hist)
static std::mutex g_grid_mu;
static bool g_smem_attr[64] = {};
static int g_coop_grid[64] = {};  // SMs of the device if it can launch cooperative sorts, else 0
static int g_coop_two[64] = {};   // two 512-thread blocks of the cooperative sort fit an SM
static int g_coop_1k[64] = {};    // one 1024-thread block of the cooperative sort fits an SM
static int g_coop_1k10[64] = {};  // ... with 1024 digit values

static void init_grids() {
  std::lock_guard<std::mutex> lock(g_grid_mu);
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  // the sort kernels' shared memory exceeds the default 48 KB: opt in on
  // every device that sorts; the cooperative sort runs one block per SM
  // (co-resident, as its grid barriers require) if the device can launch
  // cooperative grids
  if (dev >= 0 && dev < 64 && !g_smem_attr[dev]) {
    cudaFuncSetAttribute(k_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(DownSmem));
    cudaFuncSetAttribute(k_sort_coop<512, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(DownSmemT<512, 256>));
    cudaFuncSetAttribute(k_sort_coop<512, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(DownSmemT<512, 512>));
    cudaFuncSetAttribute(k_sort_coop<1024, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(DownSmemT<1024, 512>));
    cudaFuncSetAttribute(k_sort_coop<1024, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(DownSmemT<1024, 1024>));
    int coop = 0, pc = 0, pc9 = 0, pc1k = 0, nsm = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pc, k_sort_coop<512, 256>, 512,
                                                  sizeof(DownSmemT<512, 256>));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pc9, k_sort_coop<512, 512>, 512,
                                                  sizeof(DownSmemT<512, 512>));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pc1k, k_sort_coop<1024, 512>, 1024,
                                                  sizeof(DownSmemT<1024, 512>));
    int pc1k10 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pc1k10, k_sort_coop<1024, 1024>, 1024,
                                                  sizeof(DownSmemT<1024, 1024>));
    g_coop_1k10[dev] = pc1k10 >= 1 ? 1 : 0;
    g_coop_grid[dev] = (coop && pc > 0 && pc9 > 0 && nsm > 0) ? nsm : 0;
    g_coop_two[dev] = pc >= 2 ? 1 : 0;
    g_coop_1k[dev] = pc1k >= 1 ? 1 : 0;
    cudaGetLastError();
    g_smem_attr[dev] = true;
  }
  if (g_sort_blocks) return;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_downsweep, kDownThreads, sizeof(DownSmem));
  if (sms < 1) sms = 1;
  if (per > kSortBlocksPerSm) per = kSortBlocksPerSm;
  g_sort_blocks = sms * (per > 0 ? per : 1);
  g_stream_blocks = sms * 8;
}

// Runs every pass of one sort.  a.blocks must be set (at most the rows of
// a.bsum).
static cudaError_t run_sort(const SortArgs &a0, cudaStream_t s, bool hist_done = false) {
  SortArgs a = a0;
  if (a.sub < 1 || a.sub > kSortSub) a.sub = kSortSub;
  if (!hist_done) k_hist<<<a.blocks, 256, 0, s>>>(a);
  k_hist_scan<<<1, 256, 0, s>>>(a);
  const unsigned scan_blocks =
      (1u << a.digit_bits) > kScanDigits ? (1u << a.digit_bits) / kScanDigits : 1u;
  for (int p = 0; p < a.passes; ++p) {
    k_upsweep<<<a.sub * a.blocks, kSortThreads, 0, s>>>(a, p);
    k_scan_blocks<<<scan_blocks, kScanThreads, 0, s>>>(a, p);
    k_downsweep<<<a.blocks, kDownThreads, sizeof(DownSmem), s>>>(a, p);
  }
  return cudaGetLastError();
}

// Shapes of the cooperative sort: one 512-thread block per SM (beside
// another kernel), two (the sort alone), one 1024-thread block, or one with
// 1024 digit values.
enum CoopShape { kCoop512x1 = 0, kCoop512x2 = 1, kCoop1024x1 = 2, kCoop1024x1d10 = 3 };

// Blocks of the cooperative sort of that shape on the current device (0:
// the multi-kernel sort is used).
static int coop_grid(int shape = kCoop512x1) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (shape == kCoop512x2) return g_coop_two[dev] ? 2 * g_coop_grid[dev] : g_coop_grid[dev];
  if (shape == kCoop1024x1 && !g_coop_1k[dev]) return 0;
  if (shape == kCoop1024x1d10 && !g_coop_1k10[dev]) return 0;
  return g_coop_grid[dev];
}

// The whole sort in one cooperative launch of G blocks of NT threads; the
// digit tables (2 x G x NBK) live in a.bsum.
template <int NT, int NBK>
static cudaError_t run_sort_coop(const SortArgs &a, int G, cudaStream_t s) {
  // the barrier word and parity 0 of the sums start at zero
  cudaError_t e = cudaSuccess;
  if (!a.extra_zeroed) {
    e = cudaMemsetAsync(a.bsum + (size_t)2 * G * NBK, 0,
                        (size_t)(64 + kCoopSumRows * NBK) * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sizeof(DownSmemT<NT, NBK>);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_sort_coop<NT, NBK>, a);
}

// One sort: cooperative when the device allows it and the table fits
// (table_rows rows of 256 counts available in a.bsum), else multi-kernel
// (hist_done: the global histograms are already in a.hist).  `shape`: the
// blocks per SM and their size.  Digit values: 512 with a.key_range, else
// 2^digit_bits rounded up to 256, 512 or 1024; 512 values run one 512- or
// 1024-thread block per SM, 1024 values one 1024-thread block, and digits of
// more than 8 bits need the cooperative sort (the multi-kernel sort's
// histograms hold 256 values).
static int sort_nbk(const SortArgs &a) {
  return a.key_range ? 512 : (a.digit_bits <= 8 ? 256 : (a.digit_bits == 9 ? 512 : 1024));
}

static int coop_shape_for(int nbk, int shape) {
  if (nbk == 1024) return kCoop1024x1d10;
  if (nbk == 512) return shape == kCoop1024x1 ? kCoop1024x1 : kCoop512x1;
  return shape == kCoop1024x1 ? kCoop512x1 : shape;
}

static bool coop_sort_ok(int shape, long long table_rows, int nbk = 256) {
  shape = coop_shape_for(nbk, shape);
  const int G = coop_grid(shape);
  return G > 0 && G <= kCoopGroup * kCoopMaxGroups && coop_table_rows(G, nbk) <= table_rows;
}

// The shape of the cooperative sort that sort_any runs for digits of nbk
// values and the requested shape, or -1 (the multi-kernel sort).
static int coop_pick(int nbk, long long table_rows, int shape) {
  if (shape == kCoop1024x1 && !coop_sort_ok(shape, table_rows, nbk)) shape = kCoop512x1;
  shape = coop_shape_for(nbk, shape);
  return coop_sort_ok(shape, table_rows, nbk) ? shape : -1;
}

// The words of a.bsum that a cooperative sort of that shape needs cleared
// before it starts (its barrier word and first parity of sums).
static uint32_t *coop_extra(uint32_t *bsum, int shape, int nbk, long long &words) {
  words = 64 + (long long)kCoopSumRows * nbk;
  return bsum + (size_t)2 * coop_grid(shape) * nbk;
}

static cudaError_t sort_any(const SortArgs &a, long long table_rows, cudaStream_t s,
                            bool hist_done = false, int shape = kCoop512x1) {
  const int nbk = sort_nbk(a);
  shape = coop_pick(nbk, table_rows, shape);
  if (shape >= 0) {
    const int G = coop_grid(shape);
    if (nbk == 1024) return run_sort_coop<1024, 1024>(a, G, s);
    if (shape == kCoop1024x1) return run_sort_coop<1024, 512>(a, G, s);
    if (nbk == 512) return run_sort_coop<512, 512>(a, G, s);
    return run_sort_coop<512, 256>(a, G, s);
  }
  if (a.digit_bits > 8) return cudaErrorInvalidValue;   // (callers fall back to 8-bit digits)
  return run_sort(a, s, hist_done);
}

// ---- exclusive scan of pair counts in depth order -> emit offsets --------
// Reduce-then-scan over the same fixed block ranges as the sort passes: the
// upsweep sums each block's counts, the downsweep adds up the sums of the
// blocks before its own and scans its range.

struct ScanArgs {
  const uint32_t *sorted_items[2];
  const uint32_t *sel;
  const uint32_t *count;            // rec_count (by item; handed on to the emit)
  uint32_t *sorted_count[2];        // the counts in depth order: the depth sort's free key
                                    //   buffer (written by the upsweep, read by the rest)
  const uint32_t *cbig;             // count | large-item flag << 31, by item slot
  const unsigned long long *n_items;
  long long capacity;
  uint32_t *offsets;
  unsigned long long *bsum;         // [G] block sums
  int blocks;
  unsigned long long *n_pairs;
  uint32_t *bigq;                   // depth positions of the items for k_emit_big
  uint32_t *big_count;
  uint2 *ranges;                    // the per-tile ranges, zeroed here for the pair sort
  long long n_ranges;
  uint32_t *clear;                  // words zeroed here for the cooperative pair sort, or null
  long long n_clear;
};

__device__ __forceinline__ uint32_t scan_n(const ScanArgs &a) {
  unsigned long long nn = *a.n_items;
  return (uint32_t)((long long)nn > a.capacity ? a.capacity : (long long)nn);
}

// Per-block pair sums in depth order.  Each visible item's count word (the
// count and the pair count's large-item flag, in a compact array that stays
// in L2 longer than the 32-byte emit records) is gathered once, by slot: the
// count is written out in depth order, so the offset downsweep and the emit
// read counts sequentially, and the flag puts the item in the queue of
// k_emit_big (which can then run beside the emit).  1024 threads per block,
// two blocks per SM: the gathers are random once the words leave L2, so many
// must be in flight.
// (Laying out the whole 32-byte emit records in depth order here, so that
// the emit would read nothing by slot, was measured slower: 10 us more at
// 1080p, the same on a 64-view batch.)
constexpr int kOffUpThreads = 1024, kOffUpUnroll = 4;

__global__ void __launch_bounds__(kOffUpThreads, 2) k_offsets_up(ScanArgs a) {
  __shared__ unsigned long long s_w[kOffUpThreads / 32];
  const uint32_t n = scan_n(a);
  const uint32_t *items = *a.sel ? a.sorted_items[1] : a.sorted_items[0];
  uint32_t *scount = *a.sel ? a.sorted_count[0] : a.sorted_count[1];
  long long p0, p1;
  block_parts(n, a.blocks, blockIdx.x, p0, p1);
  const long long k0 = p0 * kSortPart;
  const long long k1 = p1 * kSortPart < (long long)n ? p1 * kSortPart : (long long)n;
  const uint32_t ltmask = (1u << (threadIdx.x & 31)) - 1u;
  unsigned long long sum = 0;
  for (long long base = k0; base < k1; base += kOffUpThreads * kOffUpUnroll) {
    uint32_t it[kOffUpUnroll], c[kOffUpUnroll];
#pragma unroll
    for (int u = 0; u < kOffUpUnroll; ++u) {
      const long long idx = base + u * kOffUpThreads + threadIdx.x;
      it[u] = idx < k1 ? items[idx] : 0xffffffffu;
    }
    // (every item of the visible range has its word: the pair count writes
    // one for each visible slot)
#pragma unroll
    for (int u = 0; u < kOffUpUnroll; ++u) c[u] = it[u] != 0xffffffffu ? a.cbig[it[u]] : 0u;
#pragma unroll
    for (int u = 0; u < kOffUpUnroll; ++u) {
      const long long idx = base + u * kOffUpThreads + threadIdx.x;
      const uint32_t cnt = c[u] & 0x7fffffffu;
      if (idx < k1) scount[idx] = cnt;
      sum += cnt;
      const bool big = idx < k1 && (c[u] >> 31) != 0u;
      const uint32_t bb = __ballot_sync(0xffffffffu, big);
      if (bb) {
        const int leader = __ffs(bb) - 1;
        uint32_t q0 = 0;
        if ((int)(threadIdx.x & 31) == leader) q0 = atomicAdd(a.big_count, (uint32_t)__popc(bb));
        q0 = __shfl_sync(0xffffffffu, q0, leader);
        if (big) a.bigq[q0 + __popc(bb & ltmask)] = (uint32_t)idx;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kOffUpThreads / 32; ++w) t += s_w[w];
    a.bsum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) k_offsets_down(ScanArgs a) {
  __shared__ unsigned long long s_w[8];
  __shared__ unsigned long long s_carry;
  const uint32_t n = scan_n(a);
  const uint32_t *scount = *a.sel ? a.sorted_count[0] : a.sorted_count[1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  long long p0, p1;
  block_parts(n, a.blocks, blockIdx.x, p0, p1);
  {
    // this block's base: the sums of the blocks before it (a few hundred
    // values, read from L2 by every block instead of a scan launch)
    unsigned long long before = 0;
    for (int r = tid; r < (int)blockIdx.x; r += 256) before += a.bsum[r];
    for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
    if (lane == 0) s_w[warp] = before;
    __syncthreads();
    if (tid == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < 8; ++w) t += s_w[w];
      s_carry = t;
    }
    __syncthreads();
  }
  for (long long part = p0; part < p1; ++part) {
    const long long base = part * kSortPart + (long long)tid * 16;
    // a thread's 16 consecutive counts: four 16-byte loads when all are in
    // range (base is a multiple of 16 items, the buffers 256-byte aligned)
    const bool whole = base + 16 <= (long long)n;
    uint32_t c[16];
    if (whole) {
      const uint4 *s4 = reinterpret_cast<const uint4 *>(scount + base);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 v = s4[q];
        c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) c[k] = base + k < (long long)n ? scount[base + k] : 0u;
    }
    unsigned long long tsum = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) tsum += c[k];
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
    unsigned long long run = s_carry + woff + incl - tsum;
    uint32_t o[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      o[k] = (uint32_t)(run > 0xffffffffull ? 0xffffffffull : run);
      run += c[k];
    }
    if (whole) {
      uint4 *o4 = reinterpret_cast<uint4 *>(a.offsets + base);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        o4[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (base + k < (long long)n) a.offsets[base + k] = o[k];
    }
    __syncthreads();
    if (tid == 0) s_carry += total;
  }
  // the last block's carry ends as the sum over all blocks
  if (tid == 0 && (int)blockIdx.x == a.blocks - 1) *a.n_pairs = s_carry;
  // empty ranges for the tiles the pair sort will not mark, and the pair
  // sort's barrier word and sums
  const long long t0 = (long long)blockIdx.x * 256 + tid, tstride = (long long)gridDim.x * 256;
  for (long long q = t0; q < a.n_ranges; q += tstride) a.ranges[q] = make_uint2(0u, 0u);
  if (a.clear)
    for (long long q = t0; q < a.n_clear; q += tstride) a.clear[q] = 0u;
}

// ---- emit (tile, item) pairs in depth order ------------------------------
struct EmitArgs {
  const uint32_t *sorted_items[2];
  const uint32_t *sel;
  const unsigned long long *n_items;
  long long item_capacity;
  const uint32_t *offsets;
  const uint32_t *count;
  const uint32_t *sorted_count[2];   // counts in depth order (see ScanArgs)
  const uint2 *rect;
  const uint32_t *view;
  const ViewDev *views;
  const uint8_t *tile_level;
  const uint8_t *rec_m;
  const unsigned long long *n_pairs;
  long long pair_capacity;
  uint32_t *pkey, *pval;
  uint32_t *bigq;                    // queue of items with more than kBigItem tiles
  uint32_t *big_count;
  uint32_t *hist;                    // pair sort histograms [passes][256]
  const float4 *supp;                // tight support records, or null (whole rectangle)
  const float2 *supp2;
  const uint4 *erec;                 // emit records of the pair count, 2 per item slot
  const uint32_t *level_rows;        // columns kept by the foveation filter, per row and level
  int tile;
  int passes, digit_bits;
  uint32_t *status;
};

constexpr int kEmitThreads = 128;

// Adds the pair sort's digits of tile id t (lanes with `on`) to the block's
// histograms; a warp whose tiles share a digit adds once.

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

// Emit of (tile, item) pairs in depth order.  Each item's kept tiles are an
// arithmetic function of its rank inside the item: rows of the rectangle
// (TABLE = false: no filter), or the row intervals of the table the pair
// count wrote (tight support and/or foveation filter).  So the pairs of a
// warp's 32 items are expanded load-balanced: lane l writes output positions
// g0 + l, g0 + l + 32, ... of the group, finds the owning item by binary
// search over the group's offsets (warp shuffles) and maps its rank to a
// tile.  Writes are coalesced; no lane loops over another lane's item.
// Everything an item needs besides its slot, offset and count (read in depth
// order) is its 32-byte emit record: one sector gathered per item.
// Items queued for k_emit_big (many tiles, or no row table) are skipped.
template <bool TABLE>
__global__ void __launch_bounds__(kEmitThreads) k_emit_expand(EmitArgs a) {
  __shared__ uint32_t sh[4][256];
  for (int q = threadIdx.x; q < 4 * 256; q += blockDim.x) (&sh[0][0])[q] = 0u;
  __syncthreads();
  unsigned long long nn = *a.n_items;
  const long long n = (long long)nn > a.item_capacity ? a.item_capacity : (long long)nn;
  const uint32_t *items = *a.sel ? a.sorted_items[1] : a.sorted_items[0];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const uint32_t dmask = (1u << a.digit_bits) - 1u;
  if (blockIdx.x == 0 && threadIdx.x == 0 && (long long)*a.n_pairs > a.pair_capacity)
    set_status(a.status, GS_ERR_CAPACITY);
  const long long warps = (long long)gridDim.x * (blockDim.x / 32);
  const long long wid = (long long)blockIdx.x * (blockDim.x / 32) + wl;
  // software pipeline over the warp's groups of 32 items: the next group's
  // slot, offset and count loads and its record gather are in flight while
  // this group's pairs are written
  const uint32_t *scount = *a.sel ? a.sorted_count[0] : a.sorted_count[1];
  auto load_item = [&](long long k, uint32_t &j, uint32_t &off, uint4 &e, uint4 &t) {
    j = 0; off = 0xffffffffu;
    e = make_uint4(0u, 0u, 0u, 0u);
    t = e;
    if (k < n) {
      j = items[k];
      off = a.offsets[k];
      if (scount[k] > 0) {
        e = a.erec[2 * (size_t)j];
        if (TABLE) t = a.erec[2 * (size_t)j + 1];   // (same sector)
      }
    }
  };
  uint32_t nj, noff;
  uint4 ne, nt;
  load_item(wid * 32 + lane, nj, noff, ne, nt);
  for (long long base = wid * 32; base < n; base += warps * 32) {
    const long long k = base + lane;
    const bool valid = k < n;
    const uint32_t j = nj, off = noff;
    const uint4 e = ne;
    const uint4 tload = nt;
    const uint32_t cnt = e.w;
    load_item(base + warps * 32 + lane, nj, noff, ne, nt);
    const uint32_t width = e.y & 0xffffu, rows = e.y >> 16;
    // items the offset upsweep queued for k_emit_big (the pair count's test,
    // taken again on the same record); the table exists iff the rectangle
    // is small
    const bool small = rows <= (uint32_t)kTableRows && width <= (uint32_t)kTableCols;
    const bool huge = valid && big_item(cnt, TABLE, small);
    // the row table as byte-packed inclusive prefixes of the row lengths
    // (at most kBigItem <= 127 pairs) and first columns: a pair's row is the
    // number of prefixes <= its rank
    uint32_t cumA = 0, cumB = 0, fstA = 0, fstB = 0;
    if (TABLE && valid && !huge && cnt > 0) {
      uint32_t run = 0;
#pragma unroll
      for (int q = 0; q < kTableRows; ++q) {
        int first, lastc;
        table_row(tload, q, first, lastc);
        run += lastc >= first ? (uint32_t)(lastc - first + 1) : 0u;
        if (q < 4) {
          cumA |= run << (8 * q);
          fstA |= (uint32_t)first << (8 * q);
        } else {
          cumB |= run << (8 * (q - 4));
          fstB |= (uint32_t)first << (8 * (q - 4));
        }
      }
    }
    // the pairs this kernel writes: the warp's items without the queued ones,
    // numbered by a warp scan (queued items take no iterations here)
    const uint32_t ce = (valid && !huge) ? cnt : 0u;
    uint32_t lincl = ce;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, lincl, o);
      if (lane >= o) lincl += v;
    }
    const uint32_t lexcl = lincl - ce;
    const uint32_t total = __shfl_sync(0xffffffffu, lincl, 31);
    for (uint32_t p0 = 0; p0 < total; p0 += 32) {
      const uint32_t lp = p0 + lane;
      // owning item: the last lane whose local start is <= lp (starts
      // ascend; a lane after it with no pairs starts beyond lp)
      int L = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const uint32_t o = __shfl_sync(0xffffffffu, lexcl, L + step);
        if (o <= lp) L += step;
      }
      const uint32_t lstart = __shfl_sync(0xffffffffu, lexcl, L);
      const uint32_t ioff = __shfl_sync(0xffffffffu, off, L);
      const uint32_t ij = __shfl_sync(0xffffffffu, j, L);
      const uint32_t corner = __shfl_sync(0xffffffffu, e.x, L);
      const uint32_t tx = __shfl_sync(0xffffffffu, e.z, L);
      uint32_t icA = 0, icB = 0, ifA = 0, ifB = 0, iw = 1;
      if (TABLE) {
        icA = __shfl_sync(0xffffffffu, cumA, L);
        icB = __shfl_sync(0xffffffffu, cumB, L);
        ifA = __shfl_sync(0xffffffffu, fstA, L);
        ifB = __shfl_sync(0xffffffffu, fstB, L);
      } else {
        iw = __shfl_sync(0xffffffffu, width, L);
      }
      const uint32_t rank = lp - lstart;
      const uint32_t pos = ioff + rank;
      bool wr = lp < total && (long long)pos < a.pair_capacity;
      uint32_t t = 0;
      if (wr) {
        uint32_t row = 0, col = 0;
        if (TABLE) {
          // row = #{q : prefix_q <= rank}, byte by byte: (128 + rank) -
          // prefix keeps its top bit iff prefix <= rank (both below 128: no
          // borrow between bytes)
          const uint32_t rb = (rank * 0x01010101u) | 0x80808080u;
          row = (uint32_t)(__popc((rb - icA) & 0x80808080u) + __popc((rb - icB) & 0x80808080u));
          const unsigned long long cum = (unsigned long long)icA | ((unsigned long long)icB << 32);
          const unsigned long long fst = (unsigned long long)ifA | ((unsigned long long)ifB << 32);
          const uint32_t prev = row ? (uint32_t)(cum >> (8 * (row - 1))) & 0xffu : 0u;
          col = ((uint32_t)(fst >> (8 * row)) & 0xffu) + (rank - prev);
          wr = row < (uint32_t)kTableRows;   // (always: rank < the item's count)
        } else {
          row = rank / iw;
          col = rank - row * iw;
        }
        t = corner + row * tx + col;
        if (wr) {
          a.pkey[pos] = t;
          a.pval[pos] = ij;
        }
      }
      hist_add_warp(sh, wr, t, a.passes, a.digit_bits, dmask, lane);
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < a.passes * 256; q += blockDim.x) {
    const uint32_t c = (&sh[0][0])[q];
    if (c) atomicAdd(&a.hist[q], c);
  }
}

// Items with more than kBigItem tiles (or no row table): the warps of the
// grid stride over the queue (no shared ticket to contend on), one item per
// warp.  The item's rows are taken 32 at a time, one row per lane (its kept
// interval: rectangle, tight support, foveation filter); a warp scan of the
// row lengths numbers the batch's pairs, which the lanes then write 32 at a
// time, each finding its row by binary search over the row starts.  Pairs
// come out row by row, columns ascending, as the item's rank order.
template <bool FOV, bool TIGHT>
__global__ void __launch_bounds__(256) k_emit_big(EmitArgs a) {
  __shared__ uint32_t sh[4][256];
  for (int q = threadIdx.x; q < 4 * 256; q += blockDim.x) (&sh[0][0])[q] = 0u;
  __syncthreads();
  const uint32_t nbig = *a.big_count;
  const uint32_t *items = *a.sel ? a.sorted_items[1] : a.sorted_items[0];
  const int lane = threadIdx.x & 31;
  const uint32_t dmask = (1u << a.digit_bits) - 1u;
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  for (uint32_t qi = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); qi < nbig; qi += warps) {
    const uint32_t k = a.bigq[qi];
    const uint32_t j = items[k];
    if (a.count[j] == 0u) continue;   // (never queued; an empty slot's rectangle is stale)
    const uint32_t off = a.offsets[k];
    const uint2 r = a.rect[j];
    const ViewDev &vd = a.views[a.view[j]];
    const int x0 = r.x & 0xffff, x1 = r.x >> 16, y0 = r.y & 0xffff, y1 = r.y >> 16;
    const int m = FOV ? (int)a.rec_m[j] : 0;
    SuppPre pre;
    if (TIGHT) pre = supp_prep(a.supp[j], a.supp2[j]);
    long long run = off;
    for (int yb = y0; yb <= y1; yb += 32) {
      // this lane's row: its kept columns [xa, xb] (one interval)
      const int y = yb + lane;
      int xa = x0, xb = x1;
      bool any = y <= y1;
      if (TIGHT && any) {
        int ia, ib;
        any = row_interval(pre, y, a.tile, ia, ib);
        xa = max(xa, ia);
        xb = min(xb, ib);
      }
      if (FOV && any) {
        int la, lb;
        level_row(a.level_rows, vd.row_base + y, m, la, lb);
        xa = max(xa, la);
        xb = min(xb, lb);
      }
      const uint32_t len = (any && xa <= xb) ? (uint32_t)(xb - xa + 1) : 0u;
      uint32_t incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const uint32_t excl = incl - len;
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      for (uint32_t p0 = 0; p0 < total; p0 += 32) {
        const uint32_t lp = p0 + lane;
        // owning row: the last lane whose start is <= lp (a later lane with
        // an empty row starts beyond lp)
        int L = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t o = __shfl_sync(0xffffffffu, excl, L + step);
          if (o <= lp) L += step;
        }
        const uint32_t rs = __shfl_sync(0xffffffffu, excl, L);
        const int rxa = __shfl_sync(0xffffffffu, xa, L);
        const long long o = run + lp;
        const bool wr = lp < total && o < a.pair_capacity;
        uint32_t t = 0;
        if (wr) {
          t = (uint32_t)(vd.tile_base + (long long)(yb + L) * vd.tx + (rxa + (int)(lp - rs)));
          a.pkey[o] = t;
          a.pval[o] = j;
        }
        hist_add_warp(sh, wr, t, a.passes, a.digit_bits, dmask, lane);
      }
      run += total;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < a.passes * 256; q += blockDim.x) {
    const uint32_t c = (&sh[0][0])[q];
    if (c) atomicAdd(&a.hist[q], c);
  }
}

// ---- per-tile ranges ------------------------------------------------------
constexpr int kRangeUnroll = 8;

__global__ void __launch_bounds__(256) k_ranges(const uint32_t *key_a, const uint32_t *key_b,
                                                const uint32_t *sel,
                                                const unsigned long long *n_pairs,
                                                long long capacity, long long tiles,
                                                uint2 *ranges, uint32_t *status) {
  unsigned long long nn = *n_pairs;
  const long long n = (long long)nn > capacity ? capacity : (long long)nn;
  const uint32_t *key = *sel ? key_b : key_a;
  const long long stride = (long long)gridDim.x * blockDim.x * kRangeUnroll;
  for (long long base = (long long)blockIdx.x * blockDim.x * kRangeUnroll; base < n;
       base += stride) {
    uint32_t k[kRangeUnroll], kp[kRangeUnroll], kn[kRangeUnroll];
#pragma unroll
    for (int u = 0; u < kRangeUnroll; ++u) {
      const long long p = base + u * blockDim.x + threadIdx.x;
      k[u] = p < n ? key[p] : 0u;
      kp[u] = (p > 0 && p < n) ? key[p - 1] : ~0u;
      kn[u] = p + 1 < n ? key[p + 1] : ~0u;
    }
#pragma unroll
    for (int u = 0; u < kRangeUnroll; ++u) {
      const long long p = base + u * blockDim.x + threadIdx.x;
      if (p >= n) continue;
      if ((long long)k[u] >= tiles) {   // never written by a consistent emit
        set_status(status, GS_ERR_CUDA);
        continue;
      }
      if (p == 0 || kp[u] != k[u]) ranges[k[u]].x = (uint32_t)p;
      if (p == n - 1 || kn[u] != k[u]) ranges[k[u]].y = (uint32_t)(p + 1);
    }
  }
}

// A side stream per device on which the pair count runs while the depth
// sort runs on the caller's stream (the count's records are first read by
// the pair offsets, the sort's by nothing the count does).  Fork and join
// are events enqueued under one lock, so concurrent callers cannot
// interleave them; both are capturable into a CUDA graph.
// Item slots up to which the pair count runs beside the depth sort (one
// 512-thread sort block per SM leaves room for it, and the count fills the
// sort's barrier waits); above, the count runs first and the sort takes
// 1024-thread blocks (both kernels are throughput bound there, and a count
// that starts first would hold the SMs the sort's grid needs).
constexpr long long kDepthOverlapMaxSlots = 1LL << 23;

struct SideStream {
  cudaStream_t st = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
static SideStream g_side[64];
static std::mutex g_side_mu;

static cudaError_t side_stream(int dev, SideStream *&out) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  SideStream &ss = g_side[dev];
  if (!ss.st) {
    cudaError_t e = cudaStreamCreateWithFlags(&ss.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  out = &ss;
  return cudaSuccess;
}

static cudaError_t depth_sort_and_count(const gs_plan *p, void *ws, const SortArgs &d,
                                        cudaStream_t s);

cudaError_t launch_bin_sort(const gs_plan *p, void *ws, cudaStream_t s) {
  Hdr *hdr = region<Hdr>(p, ws, R_HDR);
  cudaError_t e;
  init_grids();
  // pair sort digit width: the requested one, else the balanced width of the
  // fewest passes of at most 8 bits; widths of 9 or 10 bits only with the
  // cooperative sort (else 8)
  const long long table_rows = (long long)p->sort_blocks * kSortSub;
  int want = p->radix_bits > 0 ? p->radix_bits : 8;
  if (want > 8 && !coop_sort_ok(kCoop512x2, table_rows, want == 9 ? 512 : 1024)) want = 8;
  int pair_passes = (p->tile_bits + want - 1) / want;
  if (pair_passes > 4) pair_passes = 4;   // histogram storage holds four passes
  const int pair_bits = (p->tile_bits + pair_passes - 1) / pair_passes;
  const int pair_nbk = pair_bits <= 8 ? 256 : (pair_bits == 9 ? 512 : 1024);
  const int pair_shape = coop_pick(pair_nbk, table_rows, kCoop512x2);
  const bool coop = pair_shape >= 0;
  const bool depth_coop =
      coop_pick(512, table_rows, p->n * p->V > kDepthOverlapMaxSlots ? kCoop1024x1 : kCoop512x1) >= 0;
  // the multi-kernel sorts' histograms start from zero (the large-item
  // queue counter is cleared by the pair count)
  if (!coop || !depth_coop) {
    e = cudaMemsetAsync(&hdr->hist[0][0][0], 0, sizeof(hdr->hist), s);
    if (e != cudaSuccess) return e;
  }
  if (p->n == 0) {
    // nothing visible: empty ranges
    e = cudaMemsetAsync(region<uint2>(p, ws, R_RANGES), 0, p->bytes[R_RANGES], s);
    return e;
  }
  // grid of the reduce-then-scan kernels, at most the rows the plan holds
  const int G = g_sort_blocks < p->sort_blocks ? g_sort_blocks : p->sort_blocks;
  uint32_t *bsum = region<uint32_t>(p, ws, R_BSUM);
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
  d.drop_max = 1;                   // (cooperative sort: invisible slots are dropped by its
                                    //  first pass; the others sort the same either way)
  d.key_range = &hdr->depth_max;    // (cooperative sort: keys relative to the visible range)
  d.sel = &hdr->sel_depth;
  d.hist = &hdr->hist[0][0][0];
  d.skip = &hdr->skip[0];
  d.bsum = bsum;
  d.blocks = G;
  d.passes = 4;
  d.digit_bits = 8;
  d.status = &hdr->status;
  {
    // sub-ranges per block so that an upsweep block counts about one
    // partition of keys (few partitions per block for small scenes)
    const long long nparts = (p->n * p->V + kSortPart - 1) / kSortPart;
    const long long q = (nparts + G - 1) / G;
    d.sub = (int)(q < 1 ? 1 : (q > kSortSub ? kSortSub : q));
  }
  e = depth_sort_and_count(p, ws, d, s);
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
  sa.sorted_count[0] = d.keys[0];    // the one of the two the depth sort did not end in
  sa.sorted_count[1] = d.keys[1];
  sa.cbig = region<uint32_t>(p, ws, R_REC_CBIG);
  sa.bsum = reinterpret_cast<unsigned long long *>(bsum + (size_t)p->sort_blocks * kSortSub * 256);
  sa.blocks = G;
  sa.n_pairs = &hdr->n_pairs;
  const bool tight = (p->flags & GS_FLAG_TIGHT) != 0;
  sa.bigq = region<uint32_t>(p, ws, R_BIGQ);
  sa.big_count = &hdr->big_count;
  sa.ranges = region<uint2>(p, ws, R_RANGES);
  sa.n_ranges = p->tiles_total;
  if (coop) sa.clear = coop_extra(bsum, pair_shape, pair_nbk, sa.n_clear);
  k_offsets_up<<<G, kOffUpThreads, 0, s>>>(sa);
  k_offsets_down<<<G, 256, 0, s>>>(sa);
  // 3. emit pairs (+ the pair sort's histograms)
  EmitArgs ea = {};
  ea.sorted_items[0] = d.vals[0];
  ea.sorted_items[1] = d.vals[1];
  ea.sel = &hdr->sel_depth;
  ea.n_items = &hdr->n_visible;
  ea.item_capacity = p->max_visible;
  ea.offsets = sa.offsets;
  ea.count = sa.count;
  ea.sorted_count[0] = sa.sorted_count[0];
  ea.sorted_count[1] = sa.sorted_count[1];
  ea.rect = region<uint2>(p, ws, R_REC_RECT);
  ea.view = region<uint32_t>(p, ws, R_REC_VIEW);
  ea.views = region<ViewDev>(p, ws, R_VIEWS);
  ea.tile_level = p->has_fov ? region<uint8_t>(p, ws, R_TILE_LEVEL) : nullptr;
  ea.rec_m = p->has_fov ? region<uint8_t>(p, ws, R_REC_M) : nullptr;
  ea.supp = tight ? region<float4>(p, ws, R_REC_SUPP) : nullptr;
  ea.supp2 = tight ? region<float2>(p, ws, R_REC_SUPP2) : nullptr;
  ea.erec = region<uint4>(p, ws, R_REC_EMIT);
  ea.level_rows = p->has_fov ? region<uint32_t>(p, ws, R_LEVEL_ROWS) : nullptr;
  ea.tile = p->tile;
  ea.n_pairs = &hdr->n_pairs;
  ea.pair_capacity = p->max_pairs;
  ea.pkey = region<uint32_t>(p, ws, R_PKEY_A);
  ea.pval = region<uint32_t>(p, ws, R_PVAL_A);
  ea.hist = &hdr->hist[1][0][0];
  // the cooperative pair sort counts its own digits: the emit's histograms
  // are only needed by the multi-kernel sort
  ea.passes = coop ? 0 : pair_passes;
  ea.digit_bits = pair_bits;
  ea.status = &hdr->status;
  ea.bigq = sa.bigq;
  ea.big_count = sa.big_count;
  // the large items (queued by the offset upsweep) on the side stream, beside
  // the emit of the others
  {
    const bool fov = ea.tile_level != nullptr;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_side_mu);
    SideStream *ss = nullptr;
    if ((e = side_stream(dev, ss)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ss->fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(ss->st, ss->fork, 0)) != cudaSuccess) return e;
    if (fov && tight) k_emit_big<true, true><<<g_stream_blocks, 256, 0, ss->st>>>(ea);
    else if (fov) k_emit_big<true, false><<<g_stream_blocks, 256, 0, ss->st>>>(ea);
    else if (tight) k_emit_big<false, true><<<g_stream_blocks, 256, 0, ss->st>>>(ea);
    else k_emit_big<false, false><<<g_stream_blocks, 256, 0, ss->st>>>(ea);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ss->join, ss->st)) != cudaSuccess) return e;
    if (fov || tight) k_emit_expand<true><<<2 * g_stream_blocks, kEmitThreads, 0, s>>>(ea);
    else k_emit_expand<false><<<2 * g_stream_blocks, kEmitThreads, 0, s>>>(ea);
    if ((e = cudaStreamWaitEvent(s, ss->join, 0)) != cudaSuccess) return e;
  }
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
  t.bsum = bsum;
  t.blocks = G;
  t.passes = pair_passes;
  t.digit_bits = pair_bits;
  t.key_bits = p->tile_bits;
  t.status = &hdr->status;
  // 5. per-tile ranges: by the cooperative sort after its last pass, else
  // by a kernel of their own
  // (the ranges were zeroed by the offset downsweep)
  uint2 *ranges = sa.ranges;
  if (coop) {
    t.ranges = ranges;
    t.n_ranges = p->tiles_total;
    t.extra_zeroed = 1;   // (by the offset downsweep)
  }
  e = sort_any(t, (long long)p->sort_blocks * kSortSub,
               s, /*hist_done=*/!coop, kCoop512x2);
  if (e != cudaSuccess) return e;
  if (!coop)
    k_ranges<<<g_stream_blocks, 256, 0, s>>>(t.keys[0], t.keys[1], &hdr->sel_pair, &hdr->n_pairs,
                                           p->max_pairs, p->tiles_total, ranges, &hdr->status);
  return cudaGetLastError();
}

static cudaError_t depth_sort_and_count(const gs_plan *p, void *ws, const SortArgs &d,
                                        cudaStream_t s) {
  const long long table_rows = (long long)p->sort_blocks * kSortSub;
  if (p->n * p->V > kDepthOverlapMaxSlots) {
    // large: the pair count, then the sort on the whole GPU
    cudaError_t e = launch_count_pairs(p, ws, s);
    if (e != cudaSuccess) return e;
    return sort_any(d, table_rows, s, false, kCoop1024x1);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_side_mu);
  SideStream *ss = nullptr;
  if ((e = side_stream(dev, ss)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(ss->fork, s)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(ss->st, ss->fork, 0)) != cudaSuccess) return e;
  if ((e = launch_count_pairs(p, ws, ss->st)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(ss->join, ss->st)) != cudaSuccess) return e;
  if ((e = sort_any(d, table_rows, s, false, kCoop512x1)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(s, ss->join, 0);
}

// ---- sort of caller keys with their indices (pruning by CE) --------------
__global__ void k_set_aux_n(Hdr *h, unsigned long long n) { h->aux_n = n; }

cudaError_t launch_sort_indices(const gs_plan *p, void *ws, const uint32_t *keys, long long n,
                                cudaStream_t s) {
  Hdr *hdr = region<Hdr>(p, ws, R_HDR);
  init_grids();
  cudaError_t e = cudaMemsetAsync(&hdr->hist[0][0][0], 0, sizeof(hdr->hist[0]), s);
  if (e != cudaSuccess) return e;
  k_set_aux_n<<<1, 1, 0, s>>>(hdr, (unsigned long long)n);
  SortArgs d = {};
  d.first_keys = keys;
  d.first_vals = nullptr;                 // values = key index
  d.keys[0] = region<uint32_t>(p, ws, R_DKEY_A);
  d.keys[1] = region<uint32_t>(p, ws, R_DKEY_B);
  d.vals[0] = region<uint32_t>(p, ws, R_DVAL_A);
  d.vals[1] = region<uint32_t>(p, ws, R_DVAL_B);
  d.count = &hdr->aux_n;
  d.capacity = p->max_visible;
  d.sel = &hdr->sel_depth;
  d.hist = &hdr->hist[0][0][0];
  d.skip = &hdr->skip[0];
  d.bsum = region<uint32_t>(p, ws, R_BSUM);
  d.blocks = g_sort_blocks < p->sort_blocks ? g_sort_blocks : p->sort_blocks;
  d.passes = 4;
  d.digit_bits = 8;
  d.no_skip = 1;                          // four passes: the result ends in buffer 0
  d.status = &hdr->status;
  return sort_any(d, (long long)p->sort_blocks * kSortSub,
                  s, false, kCoop512x2);
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
// library holds that array (12,587,264 bytes: a 4,352-byte header, 8 MiB of
// temporary keys and values, a 4 MiB block table) until the process exits.
// --------------------------------------------------------------------------
namespace {

constexpr long long kStaticMax = GS_STATIC_SORT_MAX_PAIRS;
constexpr int kStaticBlocks = 1024;   // rows of the block-count table

struct StaticHdr {
  unsigned long long count;
  uint32_t hist[4][256];
  uint32_t skip[4];
  uint32_t sel;
  uint32_t status;
};

constexpr size_t kStaticHdrBytes = (sizeof(StaticHdr) + 255) & ~size_t(255);
constexpr size_t kStaticTmpBytes = 2 * sizeof(uint32_t) * (size_t)kStaticMax;   // keys + values
constexpr size_t kStaticBsumBytes = 256 * sizeof(uint32_t) * kSortSub * (size_t)kStaticBlocks;
constexpr size_t kStaticBytes = kStaticHdrBytes + kStaticTmpBytes + kStaticBsumBytes;
static_assert(kStaticBytes == 12587264, "the documented footprint of the static scratch");

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
  uint32_t *bsum = reinterpret_cast<uint32_t *>(base + kStaticHdrBytes + kStaticTmpBytes);
  init_grids();
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
  a.bsum = bsum;
  a.blocks = g_sort_blocks < kStaticBlocks ? g_sort_blocks : kStaticBlocks;
  a.no_skip = 1;
  a.status = &h->status;
  return sort_any(a, (long long)kStaticBlocks * kSortSub,
                  stream, false, kCoop512x2) == cudaSuccess
             ? GS_OK
             : GS_ERR_CUDA;
}

// Status word of the last gs_sort_pairs_static on the current device (a
// bounded wait of the sort that gave up leaves GS_ERR_TIMEOUT there).
extern "C" gs_status gs_sort_pairs_static_status(uint32_t *host_status, cudaStream_t stream) {
  using namespace gs;
  if (!host_status) return GS_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GS_ERR_CUDA;
  unsigned char *base;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    base = g_static_ptr[dev];
  }
  *host_status = GS_OK;
  if (!base) return GS_OK;   // no sort ran on this device
  const size_t off = offsetof(StaticHdr, status);
  if (cudaMemcpyAsync(host_status, base + off, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                      stream) != cudaSuccess)
    return GS_ERR_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return GS_ERR_CUDA;
  return (gs_status)*host_status;
}

// Whether the sorts run as one cooperative launch each on the current device.
extern "C" int32_t gs_sort_is_cooperative(void) {
  gs::init_grids();
  return gs::coop_grid() > 0 ? 1 : 0;
}
