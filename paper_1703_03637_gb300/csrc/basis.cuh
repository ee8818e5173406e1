// Device-side basis decode / rank of the restricted Hilbert space (section 3.1).
//
// A sector configuration s (n_ones set bits out of L + H) is split into a high part
// hi = s >> L and a low part lo = s & (2^L - 1).  Its row is
//     rank(s) = hi_off[hi] + lo_rank[lo],
// where hi_off[hi] counts the sector states whose high part is smaller than hi and
// lo_rank[lo] is the rank of lo among the L-bit strings with the same popcount: the
// split-half lookup of Lin / TITPACK that the paper uses for its reverse lookup.
// Row -> configuration goes the other way: hi is the largest value with hi_off[hi] <= r
// (binary search; a non-empty block always wins ties) and lo is entry r - hi_off[hi] of
// the ascending list of L-bit strings with popcount n_ones - popcount(hi).
#pragma once

#include "common.cuh"

namespace hphi {

__device__ __forceinline__ uint64_t sector_rank(const SectorTables& t, uint64_t s) {
  const uint64_t hi = s >> t.L;
  const uint32_t lo = (uint32_t)(s & ((1ull << t.L) - 1ull));
  return __ldg(t.hi_off + hi) + (uint64_t)__ldg(t.lo_rank + lo);
}

// Largest hi in [lo_hi, up_hi] with hi_off[hi] <= r.
__device__ __forceinline__ uint64_t sector_find_hi(const SectorTables& t, uint64_t r, uint64_t lo_hi,
                                                   uint64_t up_hi) {
  while (lo_hi < up_hi) {
    const uint64_t mid = (lo_hi + up_hi + 1) >> 1;
    if (__ldg(t.hi_off + mid) <= r) lo_hi = mid;
    else up_hi = mid - 1;
  }
  return lo_hi;
}

__device__ __forceinline__ uint64_t sector_state_in(const SectorTables& t, uint64_t r, uint64_t hi) {
  const uint64_t j = r - __ldg(t.hi_off + hi);
  const int p = t.n_ones - __popcll(hi);
  const uint32_t lo = __ldg(t.lo_list + __ldg(t.lo_list_off + p) + j);
  return (hi << t.L) | (uint64_t)lo;
}

__device__ __forceinline__ uint64_t sector_state(const SectorTables& t, uint64_t r) {
  const uint64_t hi = sector_find_hi(t, r, 0, (1ull << t.H) - 1ull);
  return sector_state_in(t, r, hi);
}

}  // namespace hphi
