// Host interface of the radix sort (radix_sort.cu).
#pragma once

#include "common.cuh"

namespace bits {

// Device scratch one sort needs; every buffer is owned by the caller.
struct RadixScratch {
  uint32_t* tmp_s;    // n keys (ping-pong buffer of the start sort)
  uint32_t* tmp_e;    // n keys (ping-pong buffer of the end sort)
  uint32_t* hist;     // 2 arrays x 4 passes x 256 digit counters
  uint32_t* status;   // radix_status_words(n) x 2 arrays x 4 passes look-back words
  uint32_t* tickets;  // 2 arrays x 4 passes tile tickets
};

// Look-back words one array needs for one pass.
size_t radix_status_words(uint32_t n);

// Sort the start words and the end words of n intervals (array of (start,
// end) pairs) into out_s / out_e.  Validates start < end (DEV_ERR_INVALID
// into d_err, returned as BITS_EINVAL); synchronises `st` once.
bits_status radix_sort_intervals(const uint2* d_b, uint32_t n, uint32_t* out_s, uint32_t* out_e,
                                 uint32_t* d_err, RadixScratch& ws, cudaStream_t st);

}  // namespace bits
