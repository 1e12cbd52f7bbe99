// Host side of the search index and the counting kernels (count.cu).
#pragma once

#include "common.cuh"
#include "db.cuh"
#include "tune.cuh"

namespace bits {

uint32_t round16(uint32_t x);

// Level sizes of the implicit 16-ary tree over n sorted keys whose top level
// holds at most 2^top_log2 - 1 entries.
void plan_levels(uint32_t n, int top_log2, LevelPlan& p);

// Fill db->lvl and write the level storage, the top images and the level-0
// padding from the sorted arrays db->bs / db->be.
bits_status build_levels(bits_db* db, cudaStream_t st);

// Zero a count's 64-bit total with a one-CTA kernel that immediately lets a
// programmatic dependent launched behind it start; that kernel waits for it
// (grid_dependency_wait) before adding to the total.
bits_status launch_zero_total(uint64_t* d_total, cudaStream_t st);

// Plain BITS count through the 16-ary levels.  Zeroes *d_total (a one-CTA
// kernel the count kernel overlaps as a programmatic dependent), then
// accumulates; d_counts may be NULL.
// tc: the tuned parameters (raise, block) to use; NULL takes them from
// count_params (pinned, tuned or default).
bits_status launch_count_search(const bits_db* db, const uint32_t* d_a, uint32_t n,
                                uint32_t* d_counts, uint64_t* d_total, cudaStream_t st,
                                const TuneCount* tc = nullptr);

// A view of the database's levels whose shared-memory top is `raise` levels
// above the default one (clamped to the levels kept), for the search kernels.
LevelIndex level_view(const bits_db* db, int raise);

}  // namespace bits
