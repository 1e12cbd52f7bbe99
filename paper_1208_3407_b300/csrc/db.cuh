// The database object behind the opaque bits_db handle.
#pragma once

#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "graph_cache.cuh"
#include "search.cuh"

// One sorted array's learned index (a two-stage recursive model): a linear
// root maps a key to one of 2^L leaves; each leaf is a linear model of the
// key's rank inside the leaf's slice of the sorted array, with the largest
// under- and over-prediction seen over that slice.
struct bits_rmi_leaf {
  uint32_t base_key;  // first key routed to the leaf (model input is key - base_key)
  uint32_t lo;        // first rank of the leaf's slice
  float slope;        // predicted rank - lo = slope * (key - base_key) + icpt
  float icpt;
  int32_t err_lo;     // min over the slice of (true rank - predicted rank)
  int32_t err_hi;     // max over the slice of (true rank - predicted rank)
  uint32_t hi;        // one past the last rank of the slice
  uint32_t pad;
};
static_assert(sizeof(bits_rmi_leaf) == 32, "one leaf is one 32-byte sector");

struct bits_rmi {
  float root_slope = 0.f;  // leaf = clamp(floor(root_slope * key + root_icpt), 0, 2^L - 1)
  float root_icpt = 0.f;
  int leaves_log2 = 0;
  bits_rmi_leaf* leaves = nullptr;  // device [2^L]
};

struct bits_mc_graph;  // cached CUDA graph of one bits_mc argument set (mc.cu)

// Sizes of the implicit 16-ary tree (see search.cuh).  The default top
// level J is the largest that fits the shared-memory cap; levels J+1 ..
// Tmax (each 16 times smaller) are also kept, with a top image each, so a
// launch may search a smaller top in shared memory and read the levels
// below it from memory instead (a tuning choice, same counts).
struct LevelPlan {
  int J = 0;                           // default top level
  int Tmax = 0;                        // highest level a launch may use as its top
  uint32_t len[bits::kMaxLevels + 1] = {};
  size_t off[bits::kMaxLevels] = {};   // word offset of level j (0 <= j < Tmax) in the level storage
  size_t level_words = 0;              // words of levels 0 .. Tmax-1, both arrays interleaved
  uint32_t top_size = 4;               // entries per array of the default top image
  uint32_t top_size_at[bits::kMaxLevels + 1] = {};  // image size of top level t (J <= t <= Tmax)
  size_t top_off[bits::kMaxLevels + 1] = {};        // word offset of that image ([2][size])
  size_t top_words = 0;                // words of all top images
};

struct bits_db {
  int device = 0;
  uint32_t n = 0;
  uint32_t* bs = nullptr;      // sorted starts, padded with 0xFFFFFFFF to 16 (device)
  uint32_t* be = nullptr;      // sorted ends, padded the same way (device)
  uint32_t* levels = nullptr;  // levels 0 .. J-1 of both arrays, interleaved by node (device)
  uint32_t* top = nullptr;     // top-level images, [2][top_size_at[t]] for J <= t <= Tmax (device)
  LevelPlan plan;
  bits::LevelIndex lvl{};      // kernel-side view of the levels
  uint32_t* err = nullptr;   // device error word (DEV_ERR_* bits)
  int method = BITS_METHOD_SEARCH;
  bool has_rmi = false;
  bits_rmi rmi[2];           // [0] starts, [1] ends
  uint2* enum_e = nullptr;   // (end, index) in start order, for enumeration (device; optional)
  void* block = nullptr;     // the one device allocation owning all of the above
  size_t block_bytes = 0;
  // Cached MC graphs keyed by the call's arguments (method, queries, n,
  // contig table, seed, shuffle range, totals) and its launch parameters,
  // at most 16.
  using McKey = std::tuple<int, const void*, uint64_t, const void*, const void*, uint32_t, uint64_t,
                           uint32_t, uint32_t, void*, int>;
  bits::GraphCache<McKey, bits_mc_graph> mc_graphs{16};
};

namespace bits {
// Synchronise `st`, read the database's device error word (and clear it if
// asked) and turn it into a status.
bits_status read_device_error(const bits_db* db, cudaStream_t st, bool clear);

// Re-sorts db->n intervals d_b into a plain database (no learned index, no
// enumeration table) and rebuilds its tree, in its own memory (capi.cu).
// Nothing is read back (every sort pass runs): the caller has checked that
// every interval has start < end.
bits_status db_rebuild(bits_db* db, const uint32_t* d_b, cudaStream_t st);
}  // namespace bits
