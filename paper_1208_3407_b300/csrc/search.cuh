// Device search primitives shared by the counting, Monte-Carlo and all-pairs
// kernels.  Every primitive returns the exact rank #(X < key) of a key in a
// sorted uint32 array X -- Algorithm 1's BSearch expressed as a count:
//     first = #(B_S < a.end)
//     last  = #(B_E <= a.start) = #(B_E < a.start + 1)   (a.start < 2^32 - 1)
// so ICount(a) = first - last (Sec. "BITS Algorithm").  Only one primitive, "count of
// elements below key", is needed.
//
// Implicit 16-ary search tree over each sorted array (built by
// k_build_levels):
//     level 0      = X itself, padded with 0xFFFFFFFF to a multiple of 16
//     level j >= 1 : L_j[i] = X[min((i+1) * 16^j, n) - 1], the last key of
//                    the i-th block of 16^j keys; also padded to 16 entries.
// L_j[i] is the last real entry of the 64-byte node L_{j-1}[16i, 16i+16),
// so if i = #(L_j < key) then #(L_{j-1} < key) = 16 i + #(node < key).
// The top level J (at most 16383 entries) lives in shared memory and is
// searched per thread; every lower level costs one 64-byte node per search,
// loaded by the four lanes of a quad (16 bytes each, fully coalesced) and
// counted with two shuffles.  Levels 0 .. J-1 are stored interleaved: node
// i of the starts' level j and node i of the ends' level j share one
// 128-byte line.  The two ranks of a query differ by its count, so for
// queries that meet few database intervals (and on the upper levels for
// nearly all) both searches read the same node index: one line, which the
// count kernel's octet descent (count.cu) reads with one load instruction,
// one memory request instead of the quad descent's two.
// Only the level-0 nodes normally come from DRAM; the levels above them
// are 1/16, 1/256, ... of the array and stay in L2.
#pragma once

#include "common.cuh"

namespace bits {

constexpr int kMaxLevels = 8;  // levels 0 .. 7: a default top J <= 5, raised by at most 2
constexpr int kMaxTop = 5;     // highest default top level (past it the top simply grows)
constexpr int kTopRaise = 2;   // levels above the default top a launch may keep in shared memory

struct LevelIndex {
  const uint32_t* x[2];               // the sorted arrays B_S, B_E (padded to 16)
  const uint32_t* il[kMaxLevels];     // level j < J of both arrays, interleaved by node:
                                      // node i of the starts at il[j] + 32 i, of the ends
                                      // at il[j] + 32 i + 16
  uint32_t len[kMaxLevels + 1];       // real entries of level j, j <= J
  const uint32_t* top;                // top level image: [2][top_size], padded with 0xFFFFFFFF
  uint32_t top_size;                  // power of two >= len[J] + 1, >= 4
  int J;
};

// L2 cache policies for the tree levels.  The upper levels (1/16, 1/256, ...
// of the array) are re-read by every search and should stay in L2; the
// level-0 chunks are touched about once per search and should not push them
// out.
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// 16-byte read-only load with an L2 cache policy.  A quad's four such loads
// cover one 64-byte node, and .L2::64B limits the line fill to that node:
// without it a random node read fills the whole 128-byte line from DRAM
// (measured: twice the DRAM bytes, the same time).
__device__ __forceinline__ uint4 ldg4_hint(const uint32_t* p, uint64_t policy) {
  uint4 v;
  asm("ld.global.nc.L2::cache_hint.L2::64B.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(policy));
  return v;
}

__device__ __forceinline__ uint32_t cnt4(const uint4 v, uint32_t key) {
  return (uint32_t)(v.x < key) + (uint32_t)(v.y < key) + (uint32_t)(v.z < key) +
         (uint32_t)(v.w < key);
}

// Shared-memory layout of the top level: each array's image (size = 2^h
// entries, sorted, the last one always padding) is stored in Eytzinger
// (breadth-first) order, node k (1 <= k < size) at index k, so that a search
// is h steps of k = 2k + (node < key): one shared load, one compare and one
// shift-add per step, and the final k - size is the rank.  Node k at depth d
// holds sorted entry ((2 (k - 2^d) + 1) << (h - 1 - d)) - 1; index 0 is
// unused.  `size` words per array.
__host__ __device__ __forceinline__ uint32_t top_words(uint32_t size) { return size; }

// #(s[0 .. size-1) < key) for both arrays' tops (starts, then ends), two
// independent searches in lock step.
__device__ __forceinline__ void top_rank2(const uint32_t* __restrict__ s_top, uint32_t size,
                                          uint32_t key_s, uint32_t key_e, uint32_t& is,
                                          uint32_t& ie) {
  const uint32_t* s_e = s_top + size;
  uint32_t ks = 1u, ke = 1u;
  for (uint32_t step = size >> 1; step; step >>= 1) {
    ks = 2u * ks + (s_top[ks] < key_s ? 1u : 0u);
    ke = 2u * ke + (s_e[ke] < key_e ? 1u : 0u);
  }
  is = ks - size;
  ie = ke - size;
}

// Cooperative copy of the two sorted top images into shared memory in
// Eytzinger order: coalesced 16-byte reads, scattered shared-memory writes.
// Sorted entry p (< size - 1) goes to node (1 << (h - 1 - t)) + ((p + 1) >> (t + 1)),
// t = trailing zeros of p + 1; entry size - 1 (padding) has no node.
__device__ __forceinline__ void load_top(uint32_t* s_top, const LevelIndex& L) {
  const uint4* src = reinterpret_cast<const uint4*>(L.top);
  const uint32_t size = L.top_size;
  const int h = 31 - __clz(size);
  for (uint32_t i = threadIdx.x; i < (2u * size) / 4u; i += blockDim.x) {
    const uint4 v = src[i];
    const uint32_t e = 4u * i;                 // element index over both arrays
    const uint32_t a = e >= size ? 1u : 0u;    // which array (4 | size: one array per uint4)
    uint32_t* dst = s_top + a * size;
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t p1 = e - a * size + (uint32_t)q + 1u;  // sorted position + 1
      const int t = __ffs(p1) - 1;
      if (t < h) dst[(1u << (h - 1 - t)) + (p1 >> (t + 1))] = w[q];
    }
  }
  if (threadIdx.x < 2) s_top[threadIdx.x * size] = kU32Max;  // unused node 0
}

// Descend the 16-ary levels for the two searches (starts, ends) of every
// thread.  A search enters at level js (resp. je) with its node index is (ie)
// there -- its rank within level js -- and leaves with its rank in X (level
// 0).  Plain search enters every search at the top level J; the learned
// index enters at the lowest node that holds its predicted window.  jmax is
// the warp-wide maximum entry level.  All 32 lanes must call it (inactive
// lanes pass js = je = 0).
__device__ __forceinline__ void quad_descend_from(const LevelIndex& L, int jmax, int js,
                                                  uint32_t& is_out, uint32_t key_s, int je,
                                                  uint32_t& ie_out, uint32_t key_e,
                                                  bool stream_level0 = true) {
  const unsigned lane = lane_id(), sub = lane & 3u, qbase = lane & ~3u;
  const uint64_t pol_last = policy_evict_last();
  const uint64_t pol_first = stream_level0 ? policy_evict_first() : pol_last;
  uint32_t is[4], ks[4], ie[4], ke[4];
  int jss[4], jes[4];
  #pragma unroll
  for (int o = 0; o < 4; ++o) {
    is[o] = __shfl_sync(0xFFFFFFFFu, is_out, qbase | o);
    ks[o] = __shfl_sync(0xFFFFFFFFu, key_s, qbase | o);
    ie[o] = __shfl_sync(0xFFFFFFFFu, ie_out, qbase | o);
    ke[o] = __shfl_sync(0xFFFFFFFFu, key_e, qbase | o);
    jss[o] = __shfl_sync(0xFFFFFFFFu, js, qbase | o);
    jes[o] = __shfl_sync(0xFFFFFFFFu, je, qbase | o);
  }
  #pragma unroll
  for (int j = kMaxLevels - 1; j >= 1; --j) {
    if (j > jmax) continue;
    const uint32_t lenj = L.len[j], lenm = L.len[j - 1];
    const uint32_t* LS = L.il[j - 1];
    const uint32_t* LE = LS + 16;
    const uint64_t pol = j == 1 ? pol_first : pol_last;
    uint4 vs[4], ve[4];
    #pragma unroll
    for (int o = 0; o < 4; ++o) {
      vs[o] = (j <= jss[o] && is[o] < lenj) ? ldg4_hint(LS + 32u * is[o] + 4u * sub, pol)
                                            : make_uint4(kU32Max, kU32Max, kU32Max, kU32Max);
      ve[o] = (j <= jes[o] && ie[o] < lenj) ? ldg4_hint(LE + 32u * ie[o] + 4u * sub, pol)
                                            : make_uint4(kU32Max, kU32Max, kU32Max, kU32Max);
    }
    #pragma unroll
    for (int o = 0; o < 4; ++o) {
      uint32_t cs = cnt4(vs[o], ks[o]), ce = cnt4(ve[o], ke[o]);
      cs += __shfl_xor_sync(0xFFFFFFFFu, cs, 1);
      ce += __shfl_xor_sync(0xFFFFFFFFu, ce, 1);
      cs += __shfl_xor_sync(0xFFFFFFFFu, cs, 2);
      ce += __shfl_xor_sync(0xFFFFFFFFu, ce, 2);
      if (j <= jss[o]) is[o] = is[o] < lenj ? 16u * is[o] + cs : lenm;
      if (j <= jes[o]) ie[o] = ie[o] < lenj ? 16u * ie[o] + ce : lenm;
    }
  }
  is_out = sub == 0 ? is[0] : sub == 1 ? is[1] : sub == 2 ? is[2] : is[3];
  ie_out = sub == 0 ? ie[0] : sub == 1 ? ie[1] : sub == 2 ? ie[2] : ie[3];
}

// Plain descent: both searches of every thread enter at the top level J.
// stream_level0: the level-0 chunks are read about once (database larger
// than L2); false when the whole database is meant to stay in L2.
__device__ __forceinline__ void quad_descend(const LevelIndex& L, uint32_t& is_out,
                                             uint32_t key_s, uint32_t& ie_out, uint32_t key_e,
                                             bool stream_level0 = true) {
  const unsigned lane = lane_id(), sub = lane & 3u, qbase = lane & ~3u;
  const uint64_t pol_last = policy_evict_last();
  const uint64_t pol_first = stream_level0 ? policy_evict_first() : pol_last;
  uint32_t is[4], ks[4], ie[4], ke[4];
  #pragma unroll
  for (int o = 0; o < 4; ++o) {
    is[o] = __shfl_sync(0xFFFFFFFFu, is_out, qbase | o);
    ks[o] = __shfl_sync(0xFFFFFFFFu, key_s, qbase | o);
    ie[o] = __shfl_sync(0xFFFFFFFFu, ie_out, qbase | o);
    ke[o] = __shfl_sync(0xFFFFFFFFu, key_e, qbase | o);
  }
  #pragma unroll
  for (int j = kMaxLevels - 1; j >= 1; --j) {
    if (j > L.J) continue;
    const uint32_t lenj = L.len[j], lenm = L.len[j - 1];
    const uint32_t* LS = L.il[j - 1];
    const uint32_t* LE = LS + 16;
    const uint64_t pol = j == 1 ? pol_first : pol_last;
    uint4 vs[4], ve[4];
    #pragma unroll
    for (int o = 0; o < 4; ++o) {
      vs[o] = is[o] < lenj ? ldg4_hint(LS + 32u * is[o] + 4u * sub, pol)
                           : make_uint4(kU32Max, kU32Max, kU32Max, kU32Max);
      ve[o] = ie[o] < lenj ? ldg4_hint(LE + 32u * ie[o] + 4u * sub, pol)
                           : make_uint4(kU32Max, kU32Max, kU32Max, kU32Max);
    }
    #pragma unroll
    for (int o = 0; o < 4; ++o) {
      uint32_t cs = cnt4(vs[o], ks[o]), ce = cnt4(ve[o], ke[o]);
      cs += __shfl_xor_sync(0xFFFFFFFFu, cs, 1);
      ce += __shfl_xor_sync(0xFFFFFFFFu, ce, 1);
      cs += __shfl_xor_sync(0xFFFFFFFFu, cs, 2);
      ce += __shfl_xor_sync(0xFFFFFFFFu, ce, 2);
      is[o] = is[o] < lenj ? 16u * is[o] + cs : lenm;
      ie[o] = ie[o] < lenj ? 16u * ie[o] + ce : lenm;
    }
  }
  is_out = sub == 0 ? is[0] : sub == 1 ? is[1] : sub == 2 ? is[2] : is[3];
  ie_out = sub == 0 ? ie[0] : sub == 1 ? ie[1] : sub == 2 ? ie[2] : ie[3];
}

// ICount of query [s, e) from its two ranks.
__device__ __forceinline__ uint32_t icount_from_ranks(uint32_t first, uint32_t last_plus,
                                                      uint32_t s, uint32_t nb) {
  const uint32_t last = (s == kU32Max) ? nb : last_plus;
  return first - last;
}

}  // namespace bits
