// Device search primitives shared by the counting, Monte-Carlo and all-pairs
// kernels.  Every primitive returns the exact rank #(B < key) of a key in a
// sorted uint32 array B -- the BSearch of Algorithm 1 expressed as a count:
//     first = #(B_S < a.end)
//     last  = #(B_E <= a.start) = #(B_E < a.start + 1)   (a.start < 2^32 - 1)
// so ICount(a) = first - last (Sec. 2.2).  Only one primitive, "count of
// elements below key", is needed.
#pragma once

#include "common.cuh"

namespace bits {

// Top tree: tree[j] (j < 2^t) is the last key of bucket j = B[j*2^k ..
// (j+1)*2^k) of the sorted array, padded with 0xFFFFFFFF past the last
// bucket.  Searching the 2^t - 1 real slots finds the bucket that holds the
// rank; a power-of-two search inside the bucket finishes it.
//
// N independent searches advance in lock step so that their loads overlap.
// Search i looks up key[i] in the start array when i is even and in the end
// array when i is odd; s_tree holds the start tree then the end tree.
template <int N>
__device__ __forceinline__ void rank_lt_tree(const uint32_t* __restrict__ s_tree, uint32_t tsz,
                                             const uint32_t* __restrict__ bs,
                                             const uint32_t* __restrict__ be, uint32_t nb, int k,
                                             const uint32_t (&key)[N], uint32_t (&pos)[N]) {
  #pragma unroll
  for (int i = 0; i < N; ++i) pos[i] = 0u;
  for (uint32_t step = tsz >> 1; step; step >>= 1) {
    #pragma unroll
    for (int i = 0; i < N; ++i) {
      const uint32_t* S = s_tree + ((i & 1) ? tsz : 0u);
      if (S[pos[i] + step - 1u] < key[i]) pos[i] += step;
    }
  }
  #pragma unroll
  for (int i = 0; i < N; ++i) pos[i] = min(pos[i] << k, nb);
  for (uint32_t step = (1u << k) >> 1; step; step >>= 1) {
    #pragma unroll
    for (int i = 0; i < N; ++i) {
      const uint32_t* B = (i & 1) ? be : bs;
      const uint32_t idx = pos[i] + step - 1u;
      const uint32_t v = idx < nb ? __ldg(B + idx) : kU32Max;
      if (v < key[i]) pos[i] += step;
    }
  }
}

// Cooperative copy of the two top trees (2 << t words) into shared memory.
__device__ __forceinline__ void load_tree(uint32_t* s_tree, const uint32_t* __restrict__ tree,
                                          uint32_t tsz) {
  const uint4* src = reinterpret_cast<const uint4*>(tree);
  uint4* dst = reinterpret_cast<uint4*>(s_tree);
  for (uint32_t i = threadIdx.x; i < (2u * tsz) / 4u; i += blockDim.x) dst[i] = src[i];
}

// ICount from the two ranks of a query (start s, end e).
__device__ __forceinline__ uint32_t icount_from_ranks(uint32_t first, uint32_t last_plus,
                                                      uint32_t s, uint32_t nb) {
  const uint32_t last = (s == kU32Max) ? nb : last_plus;
  return first - last;
}

}  // namespace bits
