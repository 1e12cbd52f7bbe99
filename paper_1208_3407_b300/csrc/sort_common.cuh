// Pieces shared by the two one-sweep radix sorts (radix_sort.cu: key/value
// pairs straight from interval pairs; sort_keys.cu: the database's keys).
#pragma once

#include "common.cuh"

namespace bits {

constexpr int kRadix = 256;   // 8-bit digits
constexpr int kPasses = 4;    // digits of a 32-bit key
constexpr int kLookAhead = 8;  // status words one look-back thread reads per round trip
// A tile's look-back word per digit: flag in the top two bits (aggregate of
// this tile only, or inclusive prefix of all tiles up to it), count below.
constexpr uint32_t kFlagAgg = 1u << 30, kFlagPre = 2u << 30, kValMask = (1u << 30) - 1;

// Words of one warp's peer table: a word per digit, 256 digits plus the
// tail's empty lanes (digit 256), padded.
constexpr int kPeerTableWords = 260;

// Lanes of the warp whose digit d equals this lane's (all 32 lanes call it
// together).  `tab` is the warp's peer table in shared memory, zero on entry
// and left zero: every lane ORs its bit into the word of its digit, reads the
// word back once all have, and clears it.  Three shared-memory operations
// per key instead of eight ballots and their bit arithmetic, which kept the
// integer pipe of the sort passes saturated.
__device__ __forceinline__ unsigned peers_by_table(uint32_t* tab, uint32_t d) {
  atomicOr(tab + d, 1u << lane_id());
  __syncwarp();
  const unsigned peers = tab[d];
  __syncwarp();
  tab[d] = 0u;
  __syncwarp();
  return peers;
}

// Exclusive scan of one value per thread over threads [0, 256); every
// thread of the block must call it.
__device__ __forceinline__ uint32_t scan256_excl(uint32_t v, uint32_t* s_w) {
  const unsigned lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t x = threadIdx.x < kRadix ? v : 0u;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (threadIdx.x < kRadix && lane == 31) s_w[w] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t t = lane < kRadix / 32 ? s_w[lane] : 0u;
    #pragma unroll
    for (int o = 1; o < kRadix / 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= (unsigned)o) t += y;
    }
    if (lane < kRadix / 32) s_w[lane] = t;
  }
  __syncthreads();
  const uint32_t r = (threadIdx.x < kRadix) ? (x - v + (w > 0 ? s_w[w - 1] : 0u)) : 0u;
  __syncthreads();
  return r;
}

// Exclusive prefix over earlier tiles of one digit's count, by decoupled
// look-back: the calling thread (one per digit) reads kLookAhead predecessor
// status words per round trip and consumes them nearest first until a tile
// that has published its inclusive prefix.  The wait is bounded: after
// kSpinLimit empty rounds it records DEV_ERR_TIMEOUT and returns what it has.
__device__ __forceinline__ uint32_t lookback_excl(const uint32_t* status, uint32_t tile,
                                                  uint32_t digit, uint32_t* err) {
  uint32_t excl = 0u, spins = 0u;
  int hi = (int)tile;  // next predecessor to consume is hi - 1
  bool done = false;
  while (!done) {
    uint32_t v[kLookAhead];
    #pragma unroll
    for (int k = 0; k < kLookAhead; ++k) {
      const int t = hi - 1 - k;
      v[k] = t >= 0 ? *(volatile const uint32_t*)(status + (size_t)t * kRadix + digit) : kFlagPre;
    }
    int used = 0;
    bool stalled = false;
    #pragma unroll
    for (int k = 0; k < kLookAhead; ++k) {
      if (done || stalled) continue;
      const uint32_t fl = v[k] & ~kValMask;
      if (fl == 0u) {
        stalled = true;
        continue;
      }
      excl += v[k] & kValMask;
      ++used;
      if (fl == kFlagPre) done = true;
    }
    hi -= used;
    if (!done && stalled) {
      if (++spins > kSpinLimit) {
        set_dev_error(err, DEV_ERR_TIMEOUT);
        break;
      }
      __nanosleep(64);
    }
  }
  return excl;
}

}  // namespace bits
