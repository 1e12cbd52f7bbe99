// Learned index over a sorted array: a two-stage recursive model (a linear
// root picks one of 2^L leaves; a linear leaf predicts the rank inside the
// leaf's slice) with per-leaf error bounds.  The model only narrows the rank
// to a window; the exact rank then comes from the 16-ary tree of search.cuh,
// entered at the lowest node whose block holds the window, so the result is
// the same count #(X < key) as the plain search, bit for bit.
//
// Exactness does not rest on the bounds: a result that lands on the edge of
// the block it was computed in is checked against its neighbour in X, and a
// failed check falls back to a plain binary search over all of X.
#pragma once

#include "db.cuh"
#include "search.cuh"

namespace bits {

struct RmiView {
  const bits_rmi_leaf* leaves[2];  // [0] starts, [1] ends
  float ra[2], rb[2];              // root: leaf = floor(ra * key + rb), clamped
  uint32_t nleaves;
};

// Root model.  The same code runs when the leaves are fitted and when they
// are searched, and every operation is monotone non-decreasing in key, so a
// leaf owns one contiguous slice of X.
__device__ __forceinline__ uint32_t rmi_root(float ra, float rb, uint32_t key, uint32_t nleaves) {
  const float f = __fmaf_rn(ra, __uint2float_rn(key), rb);
  int l = __float2int_rd(f);
  l = max(l, 0);
  l = min(l, (int)nleaves - 1);
  return (uint32_t)l;
}

// Leaf model: predicted rank of key inside the leaf's slice, in [0, cnt].
__device__ __forceinline__ int32_t rmi_predict(float slope, float icpt, uint32_t base,
                                               uint32_t cnt, uint32_t key) {
  const float x = __ll2float_rn((long long)key - (long long)base);
  const float p = fmaxf(__fmaf_rn(slope, x, icpt), 0.0f);
  const int r = __float2int_rn(fminf(p, 2147483520.0f));
  return min(r, (int)cnt);
}

// Window [wl, wh] of ranks that holds #(X < key) if the leaf's bounds hold.
__device__ __forceinline__ void rmi_window(const RmiView& R, int a, uint32_t key, uint32_t n,
                                           uint32_t& wl, uint32_t& wh) {
  const uint32_t l = rmi_root(R.ra[a], R.rb[a], key, R.nleaves);
  const uint4* rec = reinterpret_cast<const uint4*>(R.leaves[a] + l);
  const uint4 r0 = __ldg(rec), r1 = __ldg(rec + 1);
  const uint32_t base = r0.x, lo = r0.y, hi = r1.z;
  const float slope = __uint_as_float(r0.z), icpt = __uint_as_float(r0.w);
  const int err_lo = (int)r1.x, err_hi = (int)r1.y;
  const uint32_t cnt = hi >= lo ? hi - lo : 0u;
  const int p = rmi_predict(slope, icpt, base, cnt, key);
  long long l64 = (long long)lo + max(0ll, (long long)p + err_lo);
  long long h64 = (long long)lo + min((long long)cnt, (long long)p + err_hi);
  l64 = max(0ll, min(l64, (long long)n));
  h64 = max(0ll, min(h64, (long long)n));
  if (h64 < l64) {  // inconsistent leaf: search everything
    l64 = 0;
    h64 = n;
  }
  wl = (uint32_t)l64;
  wh = (uint32_t)h64;
}

// Lowest level j (1..J) whose block of 16^j ranks holds [wl, wh] strictly
// inside (touching only the ends of X); J + 1 if none does.
__device__ __forceinline__ int rmi_entry_level(int J, uint32_t wl, uint32_t wh, uint32_t n) {
  for (int j = 1; j <= J; ++j) {
    const uint32_t sh = 4u * (uint32_t)j;
    const uint64_t bstart = (uint64_t)(wl >> sh) << sh;
    const uint64_t bend = min((unsigned long long)(bstart + (1ull << sh)), (unsigned long long)n);
    const bool lo_ok = wl > bstart || wl == 0u;
    const bool hi_ok = (uint64_t)wh < bend || ((uint64_t)wh == n && bend == n);
    if (lo_ok && hi_ok) return j;
  }
  return J + 1;
}

// Key k of sorted array a (0: starts, 1: ends), read from the interleaved
// level 0 the descents use (so the check below touches the same lines), or
// from the plain array when no level is stored (J = 0).
__device__ __forceinline__ uint32_t level0_key(const LevelIndex& L, int a, uint32_t k) {
  return L.J > 0 ? __ldg(L.il[0] + 32u * (k >> 4) + 16u * (uint32_t)a + (k & 15u))
                 : __ldg(L.x[a] + k);
}

// #(X_a < key) by a binary search over ranks [lo, lo + len).
__device__ __forceinline__ uint32_t level0_lower_bound(const LevelIndex& L, int a, uint32_t lo,
                                                       uint32_t len, uint32_t key) {
  while (len > 0) {
    const uint32_t half = len >> 1;
    if (level0_key(L, a, lo + half) < key) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo;
}

// Finish one search of array a: r is the descent's result for entry level
// j (<= J), or unused when j > J (then the window is searched here).  Checks
// the block edges and falls back to a full binary search when a check fails.
__device__ __forceinline__ uint32_t rmi_finish(const LevelIndex& L, int a, uint32_t n,
                                               uint32_t key, int j, int J, uint32_t r,
                                               uint32_t wl, uint32_t wh) {
  uint32_t edge_lo, edge_hi;
  if (j > J) {
    r = level0_lower_bound(L, a, wl, wh - wl, key);
    edge_lo = wl;
    edge_hi = wh;
  } else {
    const uint32_t sh = 4u * (uint32_t)j;
    edge_lo = (wl >> sh) << sh;
    edge_hi = (uint32_t)min((unsigned long long)edge_lo + (1ull << sh), (unsigned long long)n);
  }
  bool ok = true;
  if (r == edge_lo && r > 0u) ok = level0_key(L, a, r - 1u) < key;
  if (ok && r == edge_hi && r < n) ok = level0_key(L, a, r) >= key;
  return ok ? r : level0_lower_bound(L, a, 0u, n, key);
}

// Both ranks of one thread's query through the learned index (all 32 lanes
// must call it).  On return rs = #(B_S < key_s), re = #(B_E < key_e).
__device__ __forceinline__ void rmi_rank2(const RmiView& R, const LevelIndex& L, uint32_t nb,
                                          uint32_t key_s, uint32_t key_e, uint32_t& rs,
                                          uint32_t& re, bool stream_level0 = true) {
  uint32_t wls, whs, wle, whe;
  rmi_window(R, 0, key_s, nb, wls, whs);
  rmi_window(R, 1, key_e, nb, wle, whe);
  const int js = rmi_entry_level(L.J, wls, whs, nb);
  const int je = rmi_entry_level(L.J, wle, whe, nb);
  const int ds = js <= L.J ? js : 0, de = je <= L.J ? je : 0;
  uint32_t is = ds ? wls >> (4 * ds) : 0u, ie = de ? wle >> (4 * de) : 0u;
  const int jmax = __reduce_max_sync(0xFFFFFFFFu, max(ds, de));
  if (jmax > 0) quad_descend_from(L, jmax, ds, is, key_s, de, ie, key_e, stream_level0);
  rs = rmi_finish(L, 0, nb, key_s, js, L.J, is, wls, whs);
  re = rmi_finish(L, 1, nb, key_e, je, L.J, ie, wle, whe);
}

}  // namespace bits
