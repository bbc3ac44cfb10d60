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

}  // namespace gs
