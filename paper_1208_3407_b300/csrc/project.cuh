// Projection of chromosome-local (optionally closed) intervals onto the
// half-open genome-wide line every other kernel works on (Sec. "BITS
// Algorithm" (projection), Sec. "Interval Set Intersection problem").
#pragma once

#include "common.cuh"

namespace bits {

// Maps n intervals into d_out (uint2 AoS).  d_chrom, d_off and d_len are
// ignored when n_contigs == 0.  Zeroes *d_n_rejected (if given) and adds the
// number of rejected rows to it.  Asynchronous; one kernel launch.
bits_status launch_project(const uint32_t* d_chrom, const uint32_t* d_start, const uint32_t* d_end,
                           uint64_t n, const uint32_t* d_off, const uint32_t* d_len,
                           uint32_t n_contigs, bool closed, uint32_t* d_out,
                           uint64_t* d_n_rejected, cudaStream_t st);

}  // namespace bits
