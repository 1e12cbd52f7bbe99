// Host side of the Monte-Carlo significance test (mc.cu).
#pragma once

#include "common.cuh"
#include "db.cuh"

namespace bits {

bits_status run_mc(bits_db* db, int method, const uint32_t* d_a, uint32_t n,
                   const uint32_t* d_contig_off, const uint32_t* d_contig_len, uint32_t n_contigs,
                   uint64_t seed, uint32_t shuffle_begin, uint32_t shuffle_end, uint64_t* d_totals,
                   uint64_t* h_observed, uint64_t* h_k_ge, double* h_pvalue, cudaStream_t st);

// Destroy the CUDA graphs cached in a database (called by bits_free).
void release_mc_graphs(bits_db* db);

}  // namespace bits
