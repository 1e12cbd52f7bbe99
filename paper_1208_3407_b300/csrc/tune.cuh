// Launch parameters the autotuner chooses (autotune.cu), and how a call
// finds them.
//
// Every parameter changes only how the work is laid out on the GPU, never a
// count: a tuned launch returns the same counts, totals and shuffle totals
// as any other.  A call takes, per parameter, the value pinned on its host
// thread by bits_set_tuning if there is one; otherwise the value the
// autotuner chose for its size class; otherwise the default.
#pragma once

#include <vector>

#include "common.cuh"

struct bits_db;

namespace bits {

// bits_count: search method (AUTO resolves it), levels above the
// database's default shared-memory top used as the top instead, threads
// per CTA of the search kernels.
struct TuneCount {
  int method = BITS_METHOD_SEARCH;
  int raise = 0;
  int block = 512;
};

// bits_mc: shuffles per work unit (threads per CTA), intervals per work
// unit, top raise (plain search only).
struct TuneMc {
  int shuffles = 256;
  int chunk = 1024;
  int raise = 0;
};

// The values allowed for each parameter (candidates of the autotuner).
constexpr int kCountBlocks[] = {256, 512};
constexpr int kMcShapes[][2] = {{256, 1024}, {128, 1024}, {256, 512}, {256, 2048}, {128, 2048}};
constexpr int kApChunks[] = {4096, 8192, 16384, 32768};

// Parameters of a count of n queries with `method` (SEARCH, RMI or
// MERGEPATH, or AUTO for the best of the built methods) without timing
// anything: pinned, else tuned for the size class, else defaults.
TuneCount count_params(const bits_db* db, int method, uint32_t n, bool counts);

// The same, but the first call of a size class that is neither pinned nor
// under stream capture times the candidates on the caller's inputs (the
// outputs are overwritten by the caller's own launch afterwards).
bits_status autotune_count(const bits_db* db, const uint32_t* d_a, uint32_t n,
                           uint32_t* d_counts, uint64_t* d_total, cudaStream_t st, int method,
                           TuneCount* out);

// Launch one count with explicit parameters (count.cu, rmi.cu, mergepath.cu).
bits_status launch_count_tuned(const bits_db* db, const TuneCount& t, const uint32_t* d_a,
                               uint32_t n, uint32_t* d_counts, uint64_t* d_total,
                               cudaStream_t st);

// Monte-Carlo parameters: pinned, else tuned, else defaults (no timing);
// *tuned tells whether the size class has a recorded choice.
TuneMc mc_params(const bits_db* db, int method, uint32_t n, bool* tuned);

// Monte-Carlo cache record of a size class (mc.cu times the candidates).
void mc_record(const bits_db* db, int method, uint32_t n, const TuneMc& t);
bool mc_pinned();

// Queries per all-pairs work unit: pinned, else the choice recorded for
// this argument shape (allpairs.cu times the candidates), else 8192.
// `kind` separates the record of bits_count_matrix ("allpairs") from that
// of bits_count_matrix_db ("allpairs_db").
int ap_chunk_params(uint64_t total_queries, uint64_t total_db, uint32_t n_db, uint32_t n_sets,
                    bool* tuned, const char* kind = "allpairs");
void ap_chunk_record(uint64_t total_queries, uint64_t total_db, uint32_t n_db, uint32_t n_sets,
                     int chunk, const char* kind = "allpairs");

// Low-level cache access shared by the tuners.
bool tune_lookup(const char* kind, int la, int lb, int flags, std::vector<int>* vals);
void tune_store(const char* kind, int la, int lb, int flags, const std::vector<int>& vals);
int ceil_log2_u64(uint64_t x);
bool stream_capturing(cudaStream_t st);

// The thread's pinned tuning (bits_set_tuning).
const bits_tuning& pinned_tuning();

}  // namespace bits
