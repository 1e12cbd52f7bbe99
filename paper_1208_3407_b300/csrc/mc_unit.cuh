// Device pieces of one Monte-Carlo work unit (Sec. "Monte Carlo Simulations"), shared by the
// single-test kernel (mc.cu) and the screen kernel over many query sets and
// databases (mc_matrix.cu).
//
// A unit is (chunk of kMcChunk intervals, block of kMcBlock shuffles).  The
// chunk is staged in shared memory with each interval's contig offset,
// length and placement range; then each thread owns one shuffle, walks the
// chunk (a broadcast read), draws one Philox4x32-10 block per interval at
// counter (interval, shuffle, set, 0), places the interval with a
// multiply-high offset and counts it with the two rank searches of the
// database.
#pragma once

#include "philox.cuh"
#include "rmi_search.cuh"
#include "search.cuh"

namespace bits {

constexpr int kMcBlock = 256;    // default shuffles per work unit (one per thread)
constexpr int kMcChunk = 1024;   // default intervals per work unit
constexpr int kMaxContigs = 4096;
static_assert(kMcChunk % kMcBlock == 0, "a chunk is staged in whole rounds of the block");
// Resident CTAs per SM of the Monte-Carlo kernels: the shared-memory top and
// staging (~45 KB a CTA) would allow five, but four with the shared-memory
// carveout fitted to them leave ~60 KB of L1 for the level-0 chunk loads,
// which measured 7 % faster.
constexpr int kMcCtasPerSm = 4;

// Contig of a position: last contig whose offset is <= pos, or -1.
__device__ __forceinline__ int contig_of(const uint32_t* s_coff, uint32_t nc, uint32_t pos) {
  uint32_t lo = 0, len = nc;  // count of offsets <= pos
  while (len > 0) {
    const uint32_t half = len >> 1;
    if (s_coff[lo + half] <= pos) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return (int)lo - 1;
}

// Stage intervals [i0, i0 + cn) of A: contig offset, length and number of
// possible starts (contig length - length + 1).  An interval that is
// inverted, lies before the first contig or crosses its contig's end sets
// `bad` and is pinned in place (range 1, length 0).  Each thread issues all
// of its loads before it uses any, so a chunk costs one memory round trip.
// Must be called by exactly BLOCK threads; CHUNK is a multiple of BLOCK.
template <int BLOCK = kMcBlock, int CHUNK = kMcChunk>
__device__ __forceinline__ void mc_stage_chunk(const uint2* __restrict__ A, uint32_t i0,
                                               uint32_t cn, const uint32_t* s_coff,
                                               const uint32_t* s_clen, uint32_t nc,
                                               uint32_t* s_off, uint32_t* s_len, uint32_t* s_rng,
                                               bool& bad) {
  static_assert(CHUNK % BLOCK == 0, "a chunk is staged in whole rounds of the block");
  constexpr int kPer = CHUNK / BLOCK;
  uint2 qs[kPer];
  #pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const uint32_t k = threadIdx.x + (uint32_t)r * BLOCK;
    qs[r] = k < cn ? A[i0 + k] : make_uint2(0u, 0u);
  }
  #pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const uint32_t k = threadIdx.x + (uint32_t)r * BLOCK;
    if (k >= cn) continue;
    const uint2 q = qs[r];
    const int c = contig_of(s_coff, nc, q.x);
    const bool ok = c >= 0 && q.y >= q.x &&
                    (unsigned long long)q.y <= (unsigned long long)s_coff[c] + s_clen[c];
    if (ok) {
      s_off[k] = s_coff[c];
      s_len[k] = q.y - q.x;
      s_rng[k] = s_clen[c] - (q.y - q.x) + 1u;
    } else {
      bad = true;
      s_off[k] = q.x;
      s_len[k] = 0u;
      s_rng[k] = 1u;
    }
  }
}

// Which shuffle and which intervals of the staged chunk a thread takes in
// shuffle block sb.  A full block gives each of the kMcBlock threads its own
// shuffle and the whole chunk.  A short block (the last one, or a call with
// fewer than kMcBlock shuffles) of ns shuffles splits the CTA into
// groups = kMcBlock / ns groups of ns threads: thread t takes shuffle t % ns
// and every groups-th interval from t / ns, so small shuffle counts still
// use the whole CTA.  The threads past groups * ns stay idle.
struct McLane {
  uint32_t s_local;  // shuffle index relative to the call's first shuffle
  uint32_t group, groups;
  bool active;
};

template <int BLOCK = kMcBlock>
__device__ __forceinline__ McLane mc_lane(uint32_t sb, uint32_t n_shuffles) {
  const uint32_t first = sb * BLOCK;
  const uint32_t ns = min((uint32_t)BLOCK, n_shuffles - first);
  McLane l;
  l.groups = BLOCK / ns;
  l.group = threadIdx.x / ns;
  l.s_local = first + threadIdx.x % ns;
  l.active = l.group < l.groups;
  return l;
}

// This thread's share of the total over the staged chunk of ICount(placed
// interval) for its shuffle s.  Every lane runs the same number of
// iterations (the tree descent is warp-cooperative); lanes without an
// interval search a dummy key and add nothing.
template <bool kRmi>
__device__ __forceinline__ unsigned long long mc_count_chunk(
    const uint32_t* s_top, const LevelIndex& L, const RmiView& R, uint32_t nb,
    const uint32_t* s_off, const uint32_t* s_len, const uint32_t* s_rng, uint32_t i0, uint32_t cn,
    const McLane& ln, uint32_t s, uint32_t set, uint32_t key0, uint32_t key1) {
  unsigned long long acc = 0ull;
  for (uint32_t kk = 0; kk < cn; kk += ln.groups) {
    const uint32_t k = kk + ln.group;
    const bool valid = ln.active && k < cn;
    const uint32_t kc = valid ? k : 0u;
    const uint32_t off = s_off[kc], rng = s_rng[kc], len = s_len[kc];
    const uint4 x = philox4x32_10(make_uint4(i0 + kc, s, set, 0u), key0, key1);
    const uint32_t start = off + philox_offset(x, rng);
    const uint32_t end = start + len;
    uint32_t rs, re;
    const uint32_t key_s = end, key_e = start + 1u;
    if (kRmi) {
      rmi_rank2(R, L, nb, key_s, key_e, rs, re, false);
    } else {
      top_rank2(s_top, L.top_size, key_s, key_e, rs, re);
      quad_descend(L, rs, key_s, re, key_e, false);
    }
    const uint32_t c = icount_from_ranks(rs, re, start, nb);
    acc += valid ? c : 0u;
  }
  return acc;
}

}  // namespace bits
