// Merge-path counting variant (mergepath.cu).
#pragma once

#include "common.cuh"
#include "db.cuh"

namespace bits {

bits_status launch_count_mergepath(const bits_db* db, const uint32_t* d_a, uint32_t n,
                                   uint32_t* d_counts, uint64_t* d_total, cudaStream_t st);

}  // namespace bits
