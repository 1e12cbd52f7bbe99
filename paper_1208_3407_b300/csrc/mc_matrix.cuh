// Host side of the Monte-Carlo screen over query sets x databases (mc_matrix.cu).
#pragma once

#include "common.cuh"
#include "db.cuh"

namespace bits {

bits_status run_mc_matrix(const bits_db* const* dbs, uint32_t n_db, const uint32_t* const* d_as,
                          const uint64_t* n_as, uint32_t n_sets, const uint32_t* d_contig_off,
                          const uint32_t* d_contig_len, uint32_t n_contigs, uint64_t seed,
                          uint32_t shuffle_begin, uint32_t shuffle_end, uint64_t* d_observed,
                          uint64_t* d_totals, bits_mc_stat* d_stats, cudaStream_t st);

// Drop the cached launch graphs that reference a database (called by bits_free).
void release_mc_matrix_graphs(const bits_db* db);

}  // namespace bits
