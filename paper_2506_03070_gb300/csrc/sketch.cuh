// sketch.cuh -- generation of one column of the sparse sign sketch S, in
// registers (Sec. 3.1.2 rejection sampling; signs as in Algorithm 3).
#pragma once
#include <limits.h>

#include "common.cuh"

namespace lsq {

// Ascending bitonic sorting network on N (power of two) register values.
template <int N>
__device__ __forceinline__ void bitonic_sort(int32_t (&c)[N]) {
#pragma unroll
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const int32_t lo = min(c[i], c[l]), hi = max(c[i], c[l]);
          if ((i & k) == 0) {
            c[i] = lo;
            c[l] = hi;
          } else {
            c[i] = hi;
            c[l] = lo;
          }
        }
      }
    }
  }
}

// Replace the slots j set in `mask` by the round-r draws of column `col`:
// Philox4x64-10 keyed (seed, 0) at counter (col, r, j/4, 0), word j%4.
template <int N>
__device__ __forceinline__ void draw_slots(uint64_t seed, uint64_t col, uint64_t r, uint64_t mask, uint64_t d,
                                           int32_t (&c)[N]) {
#pragma unroll
  for (int q = 0; q < N / 4; ++q) {
    if ((mask >> (4 * q)) & 0xFull) {
      const U64x4 blk = philox4x64_10(col, r, (uint64_t)q, 0ull, seed, 0ull);
#pragma unroll
      for (int w = 0; w < 4; ++w)
        if ((mask >> (4 * q + w)) & 1ull) c[4 * q + w] = word_to_index(blk.w[w], d);
    }
  }
}

// Column `col` of S: zeta distinct indices in [0, d), ascending, in c[0..zeta)
// (c[zeta..N) = INT_MAX), and the sign word (bit k set -> slot k is +1).
// Steps: (i) draw zeta indices with replacement; (ii) sort and compare
// neighbours; (iii) for every equal neighbour pair (j, j+1) redraw slot j;
// (iv) repeat (ii)-(iii) until all differ.  Returns the number of redraw
// rounds, or -1 past the round cap.
template <int N>
__device__ __forceinline__ int sketch_column(uint64_t seed, uint64_t col, uint64_t d, int zeta, int32_t (&c)[N],
                                             uint64_t& signs) {
#pragma unroll
  for (int j = 0; j < N; ++j) c[j] = INT_MAX;
  const uint64_t all = zeta >= 64 ? ~0ull : ((1ull << zeta) - 1ull);
  draw_slots<N>(seed, col, 0ull, all, d, c);
  bitonic_sort<N>(c);
  int r = 0;
  for (;;) {
    uint64_t dup = 0;
#pragma unroll
    for (int j = 0; j + 1 < N; ++j)
      if (j + 1 < zeta && c[j] == c[j + 1]) dup |= 1ull << j;
    if (dup == 0) break;
    if (++r > kMaxRounds) {
      r = -1;
      break;
    }
    draw_slots<N>(seed, col, (uint64_t)r, dup, d, c);
    bitonic_sort<N>(c);
  }
  signs = philox4x64_10(col, 0ull, 0ull, 1ull, seed, 0ull).w[0];
  return r;
}

}  // namespace lsq
