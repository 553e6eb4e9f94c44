// A 32-ary min-tree over an LCP array (level 0 is the array itself, each
// further level holds the minima of 32 entries of the level below) and the
// "previous smaller value" query on it.  Used for the LCP-interval left end
// of a sub-string: 1 + max{ j < k : LCP[j] < l }.
#pragma once

#include <stdint.h>

#include "apo_internal.cuh"

namespace apo {

constexpr int kMaxTree = 8;

struct MinTree {
  const uint32_t *lv[kMaxTree];
  uint32_t cnt[kMaxTree];
  int nlev;
};

__global__ void k_min32(const uint32_t *__restrict__ in, uint32_t nin, uint32_t *__restrict__ out,
                        uint32_t nout);

// Largest j < k with level-0 value < l, or -1.  Walks up one level while no
// smaller value lies to the left within the current 32-block, then down
// into the nearest block that has one.
__device__ __forceinline__ long long prev_less(const MinTree &T, uint32_t k, uint32_t l, uint32_t *err) {
  uint32_t x = k;
  for (int lev = 0; lev < T.nlev; ++lev) {
    const uint32_t *a = T.lv[lev];
    const uint32_t lo = x & ~31u;
    for (uint32_t j = x; j > lo;) {
      --j;
      if (a[j] < l) {
        uint32_t idx = j;
        for (int d = lev; d > 0; --d) {
          const uint32_t *b = T.lv[d - 1];
          const uint32_t first = idx * 32;
          uint32_t jj = min(first + 32, T.cnt[d - 1]);
          while (jj > first && b[jj - 1] >= l) --jj;
          if (jj == first) {
            atomicExch(err, kDevRange);
            return -1;
          }
          idx = jj - 1;
        }
        return idx;
      }
    }
    if (lo == 0) return -1;
    x = lo >> 5;
  }
  return -1;
}

// Builds the levels above `lcp` (n entries) from the context's arena.
int build_min_tree(apo_ctx *c, const uint32_t *lcp, uint32_t n, MinTree *T, cudaStream_t s);

}  // namespace apo
