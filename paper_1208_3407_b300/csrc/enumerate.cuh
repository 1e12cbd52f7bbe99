// Enumeration of intersecting pairs (enumerate.cu).
#pragma once

#include "common.cuh"
#include "db.cuh"

namespace bits {

// (end, index) pairs of the database in start order, from the start-sorted
// indices d_idx of the interval pairs d_b.
bits_status launch_enum_gather(const uint32_t* d_b, const uint32_t* d_idx, uint32_t n, uint2* d_out,
                               cudaStream_t st);

// offsets[i] = first pair of query i, offsets[n] = number of pairs.
bits_status run_enumerate_offsets(const bits_db* db, const uint32_t* d_a, uint32_t n,
                                  uint64_t* d_offsets, cudaStream_t st);

// Writes (query, database index) pairs at the offsets; needs db->enum_e.
bits_status run_enumerate_pairs(const bits_db* db, const uint32_t* d_a, uint32_t n,
                                const uint64_t* d_offsets, uint32_t* d_pairs, cudaStream_t st);

}  // namespace bits
