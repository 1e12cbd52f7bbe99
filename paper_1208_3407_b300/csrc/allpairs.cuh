// All-pairs count matrix (allpairs.cu).
#pragma once

#include "common.cuh"
#include "db.cuh"

namespace bits {

bits_status run_count_matrix(const bits_db* const* dbs, uint32_t n_db,
                             const uint32_t* const* d_as, const uint64_t* n_as, uint32_t n_sets,
                             uint64_t* d_matrix, cudaStream_t st);

// The matrix from databases on both sides (bits_count_matrix_db).
bits_status run_count_matrix_db(const bits_db* const* a_dbs, uint32_t n_a,
                                const bits_db* const* b_dbs, uint32_t n_b, uint64_t* d_matrix,
                                cudaStream_t st);

// Forget the cached all-pairs graphs that use `db` (called by bits_free).
void release_matrix_graphs(const bits_db* db);

}  // namespace bits
