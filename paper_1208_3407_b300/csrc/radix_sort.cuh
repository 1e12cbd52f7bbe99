// Host interface of the radix sort (radix_sort.cu).
#pragma once

#include "common.cuh"

namespace bits {

// Device scratch one sort needs; every buffer is owned by the caller.
struct RadixScratch {
  uint32_t* tmp_s;    // n keys (ping-pong buffer of the first array)
  uint32_t* tmp_e;    // n keys (ping-pong buffer of the second array)
  uint32_t* hist;     // kRadixHistWords: 2 arrays x 4 passes x 256 digit counters + 1 flag
  uint32_t* status;   // radix_status_words(n) x 2 arrays x 4 passes look-back words
  uint32_t* tickets;  // 2 arrays x 4 passes tile tickets
};

constexpr size_t kRadixHistWords = 2 * 4 * 256 + 64;

// Keys a one-sweep tile holds (threads x keys per thread); the look-back
// table has 256 words per tile, array and pass.
constexpr uint32_t kRadixTileKeys = 8192;
constexpr size_t radix_status_words_max(uint32_t n) {
  return (size_t)((n + kRadixTileKeys - 1) / kRadixTileKeys) * 256;
}

// One of the two arrays a sort produces.  Its keys come from the interval
// pairs: word `comp` (0 start, 1 end) plus `add`.  With out_vals set, the
// values are the intervals' indices, top bit set for inverted intervals when
// flag_inverted is set.
struct SortSpec {
  int comp = 0;
  uint32_t add = 0;
  int flag_inverted = 0;
  uint32_t* out_keys = nullptr;
  uint32_t* out_vals = nullptr;  // NULL: keys only (must agree for both specs)
  uint32_t* tmp_keys = nullptr;
  uint32_t* tmp_vals = nullptr;
};

// Look-back words one array needs for one pass.
size_t radix_status_words(uint32_t n);

// Sort the two keys of n intervals into spec[0] and spec[1].  validate = 0:
// every interval must have start < end (else BITS_EINVAL); validate = 1:
// intervals with end < start are reported through *any_inverted.  Reads the
// histograms on the host (synchronises `st` once).
bits_status radix_sort_pairs(const uint2* d_src, uint32_t n, const SortSpec spec[2], int validate,
                             uint32_t* d_err, RadixScratch& ws, cudaStream_t st,
                             bool* any_inverted);

// The database sort: starts into out_s, ends into out_e (keys only).  With
// read_back (the default) it reads the digit histograms on the host
// (synchronising `st` once), skips passes whose digit is the same for every
// key and returns BITS_EINVAL for an interval with end <= start; without it
// nothing is read back, every pass runs and such an interval only sets
// d_err (for inputs already checked).
bits_status radix_sort_intervals(const uint2* d_b, uint32_t n, uint32_t* out_s, uint32_t* out_e,
                                 uint32_t* d_err, RadixScratch& ws, cudaStream_t st,
                                 bool read_back = true);

}  // namespace bits
