// lookback.cuh -- decoupled look-back prefix propagation with bounded waits.
//
// A partition publishes its aggregate, then walks back over its
// predecessors' slots until it meets an inclusive prefix.  Partitions are
// numbered by an atomic ticket, so a partition only ever waits on
// partitions that an already running block owns.  Every wait is bounded:
// after kSpinLimit polls the status word gets GS_ERR_TIMEOUT and the walk
// stops (the result is then wrong but every later index is clamped, so no
// access leaves its buffer).
#pragma once

#include <stdint.h>

#include "gs_internal.cuh"

namespace gs {

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Relaxed load: a look-back slot carries its own count in the same 64-bit
// word as its flag, so no other data needs ordering after reading it.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Single value, called by one thread of the partition's block.  Returns the
// exclusive prefix of `agg` over partitions 0..part-1.
__device__ __forceinline__ unsigned long long lookback_single(unsigned long long *slots,
                                                              uint32_t part,
                                                              unsigned long long agg,
                                                              uint32_t *status) {
  if (part == 0) {
    st_release_u64(&slots[0], kFlagPre | agg);
    return 0ull;
  }
  st_release_u64(&slots[part], kFlagAgg | agg);
  unsigned long long excl = 0;
  long long q = (long long)part - 1;
  int spins = 0;
  while (q >= 0) {
    unsigned long long w = ld_acquire_u64(&slots[q]);
    unsigned long long f = w >> 62;
    if (f == 2ull) {
      excl += w & kValMask;
      break;
    }
    if (f == 1ull) {
      excl += w & kValMask;
      --q;
      continue;
    }
    if (++spins > kSpinLimit) {
      set_status(status, GS_ERR_TIMEOUT);
      break;
    }
    __nanosleep(32);
  }
  st_release_u64(&slots[part], kFlagPre | (excl + agg));
  return excl;
}

// Warp-cooperative single value: called by all 32 lanes of one warp.  Each
// step reads 32 predecessors at once, sums the aggregates after the
// nearest inclusive prefix, and moves 32 partitions back until a prefix is
// found.  Returns the exclusive prefix (same value in every lane).
__device__ __forceinline__ unsigned long long lookback_single_warp(unsigned long long *slots,
                                                                   uint32_t part,
                                                                   unsigned long long agg,
                                                                   uint32_t *status) {
  const int lane = threadIdx.x & 31;
  if (part == 0) {
    if (lane == 0) st_release_u64(&slots[0], kFlagPre | agg);
    return 0ull;
  }
  if (lane == 0) st_release_u64(&slots[part], kFlagAgg | agg);
  unsigned long long excl = 0;
  long long hi = (long long)part - 1;   // newest predecessor not yet summed
  int spins = 0;
  while (hi >= 0) {
    const long long q = hi - lane;      // lane 0 = newest
    unsigned long long w = q >= 0 ? ld_relaxed_u64(&slots[q]) : (kFlagPre | 0ull);
    const unsigned long long f = w >> 62;
    const uint32_t pre = __ballot_sync(0xffffffffu, f == 2ull);
    const uint32_t notready = __ballot_sync(0xffffffffu, f == 0ull);
    // lanes up to (and including) the nearest prefix, if no unready slot
    // comes before it
    const int first_pre = pre ? __ffs(pre) - 1 : 32;
    const int first_nr = notready ? __ffs(notready) - 1 : 32;
    if (first_nr < first_pre) {
      // sum the ready aggregates in front of the gap, then wait there
      unsigned long long v = lane < first_nr ? (w & kValMask) : 0ull;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      excl += v;
      hi -= first_nr;
      if (++spins > kSpinLimit) {
        if (lane == 0) set_status(status, GS_ERR_TIMEOUT);
        break;
      }
      if (first_nr == 0) __nanosleep(32);
      continue;
    }
    unsigned long long v = lane <= first_pre ? (w & kValMask) : 0ull;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (first_pre < 32) break;
    hi -= 32;
  }
  if (lane == 0) st_release_u64(&slots[part], kFlagPre | (excl + agg));
  return excl;
}

}  // namespace gs
