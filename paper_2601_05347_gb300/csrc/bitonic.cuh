// bitonic.cuh -- block-wide bitonic sorting network in which every
// compare-exchange moves the smaller element to the lower index: each merge
// stage first compares element t with its mirror inside the current block of
// size kk, then runs half-cleaners.  Positions at or past `len` behave as
// +infinity and are never read or written, so any length sorts in place.
// Call with every thread of the block.
#pragma once
#include <stdint.h>

namespace psi {

template <class Less, class Swap>
__device__ void bitonic_ascending(int64_t len, Less less, Swap swap) {
  int64_t P = 1;
  while (P < len) P <<= 1;
  for (int64_t kk = 2; kk <= P; kk <<= 1) {
    for (int64_t t = threadIdx.x; t < P; t += blockDim.x) {
      if (t & (kk >> 1)) continue;
      const int64_t u = t ^ (kk - 1);
      if (u < len && less(u, t)) swap(t, u);
    }
    __syncthreads();
    for (int64_t jj = kk >> 2; jj > 0; jj >>= 1) {
      for (int64_t t = threadIdx.x; t < P; t += blockDim.x) {
        if (t & jj) continue;
        const int64_t u = t + jj;
        if (u < len && less(u, t)) swap(t, u);
      }
      __syncthreads();
    }
  }
}

}  // namespace psi
