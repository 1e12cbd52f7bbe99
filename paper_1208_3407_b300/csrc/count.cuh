// Host launchers of the counting kernels.
#pragma once

#include "common.cuh"
#include "db.cuh"

namespace bits {

// Plain BITS count: top tree in shared memory + binary search in the bucket.
// Zeroes *d_total, then accumulates; d_counts may be NULL.
bits_status launch_count_search(const bits_db* db, const uint32_t* d_a, uint32_t n,
                                uint32_t* d_counts, uint64_t* d_total, cudaStream_t st);

// Method the autotuner picks for an AUTO count of n queries.
int choose_count_method(const bits_db* db, uint32_t n);

}  // namespace bits
