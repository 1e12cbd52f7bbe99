// The database object behind the opaque bits_db handle.
#pragma once

#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "common.cuh"

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

struct bits_db {
  int device = 0;
  uint32_t n = 0;
  uint32_t* bs = nullptr;    // sorted starts (device)
  uint32_t* be = nullptr;    // sorted ends (device)
  uint32_t* tree = nullptr;  // start tree [2^t] then end tree [2^t] (device)
  int tree_log2 = 12;        // t
  int bucket_log2 = 0;       // k: every bucket holds 2^k ranks
  uint32_t* err = nullptr;   // device error word (DEV_ERR_* bits)
  int method = BITS_METHOD_SEARCH;
  bool has_rmi = false;
  bits_rmi rmi[2];           // [0] starts, [1] ends
  void* block = nullptr;     // the one device allocation owning all of the above
  size_t block_bytes = 0;
  // Cached MC graphs keyed by the call's arguments.
  std::mutex mu;
  std::map<std::tuple<int, const void*, uint64_t, const void*, const void*, uint32_t, uint64_t,
                      uint32_t, uint32_t, void*, void*>,
           std::shared_ptr<bits_mc_graph>>
      mc_graphs;
};
