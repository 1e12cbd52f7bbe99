// Learned index (two-stage recursive model) over one sorted array (rmi.cu).
#pragma once

#include "common.cuh"
#include "db.cuh"
#include "rmi_search.cuh"
#include "tune.cuh"

namespace bits {

// Fit the root and the 2^L leaves of `rmi` on the sorted keys, on the device.
bits_status rmi_build(const uint32_t* keys, uint32_t n, bits_rmi& rmi, cudaStream_t st);

// Kernel-side view of a database's two learned indexes.
RmiView rmi_view(const bits_db* db);

// bits_count through the learned index of both sorted arrays; tc: the tuned
// threads per CTA (NULL: from count_params).
bits_status launch_count_rmi(const bits_db* db, const uint32_t* d_a, uint32_t n,
                             uint32_t* d_counts, uint64_t* d_total, cudaStream_t st,
                             const TuneCount* tc = nullptr);

}  // namespace bits
