// Warp-wide search of a non-decreasing int64 array (the batched tile walk's
// message weight offsets).
#pragma once

#include <cstdint>

namespace gb64 {

// Largest j in [0, nmsg) with off[j] <= x (off non-decreasing, off[0] <= x
// < off[nmsg]). The whole warp searches: each round its 32 lanes probe 32
// evenly spaced offsets and the count of those <= x narrows the interval
// 33-fold (4 dependent loads for 10^5 messages, not 17).
__device__ __forceinline__ int64_t owner_of_warp(const int64_t* off, int64_t nmsg, int64_t x,
                                                 uint32_t lane) {
  int64_t lo = 0, hi = nmsg;  // invariant: off[lo] <= x < off[hi]
  while (hi - lo > 1) {
    const int64_t span = hi - lo;
    // probes lo < p_0 <= p_1 <= ... <= p_31 < hi
    const int64_t p = lo + 1 + (span - 1) * (int64_t)lane / 32;
    const uint32_t le = __ballot_sync(0xFFFFFFFFu, __ldg(off + p) <= x);
    const int c = __popc(le);  // the probes <= x are lanes [0, c)
    const int64_t below = __shfl_sync(0xFFFFFFFFu, p, c > 0 ? c - 1 : 0);
    const int64_t above = __shfl_sync(0xFFFFFFFFu, p, c < 32 ? c : 31);
    if (c > 0) lo = below;
    if (c < 32) hi = above;
  }
  return lo;
}

}  // namespace gb64
