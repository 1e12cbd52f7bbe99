// Batched summary of Monte-Carlo tests (mc_stats.cu).
#pragma once

#include "common.cuh"

namespace bits {

// d_totals: n_tests rows of n_shuffles uint64; d_observed: uint64[n_tests];
// d_stats: bits_mc_stat[n_tests].  One launch, asynchronous.
bits_status launch_mc_summary(const uint64_t* d_totals, uint32_t n_shuffles, uint32_t n_tests,
                              const uint64_t* d_observed, bits_mc_stat* d_stats, cudaStream_t st);

}  // namespace bits
