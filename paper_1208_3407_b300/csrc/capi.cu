// C ABI entry points (include/bits.h) and the host runtime around them:
// database construction and ownership, argument checking, method dispatch,
// error reporting and the launch counter.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "count.cuh"
#include "db.cuh"
#include "mc.cuh"
#include "radix_sort.cuh"
#include "rmi.cuh"
#include "allpairs.cuh"
#include "mergepath.cuh"
#include "project.cuh"
#include "mc_stats.cuh"
#include "mc_matrix.cuh"
#include "enumerate.cuh"

namespace bits {
namespace {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
std::mutex g_sm_mu;
std::vector<int> g_sm_count;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }
void count_launch(uint32_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void uncount_launch(uint64_t k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }

int sm_count() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_sm_mu);
  if ((int)g_sm_count.size() <= dev) g_sm_count.resize(dev + 1, 0);
  if (g_sm_count[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    g_sm_count[dev] = v > 0 ? v : 1;
  }
  return g_sm_count[dev];
}

int kernel_blocks_per_sm(const void* kernel, int block, size_t smem, int cap) {
  // Per (device, kernel): the largest dynamic shared-memory limit set so far
  // (the limit only grows, so every earlier launch size stays valid), the
  // shared-memory size the carveout was last fitted to, and the occupancy
  // per (block, smem, cap).
  struct State {
    size_t limit = 0;
    size_t carve_for = ~size_t(0);
    std::map<std::tuple<int, size_t, int>, int> occ;
  };
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, State> states;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  State& S = states[std::make_pair(dev, kernel)];
  if (smem > S.limit) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    S.limit = smem;
  }
  const auto key = std::make_tuple(block, smem, cap);
  auto it = S.occ.find(key);
  int b = 0;
  if (it != S.occ.end()) {
    b = it->second;
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, block, smem);
    b = std::max(1, b);
    if (cap > 0) b = std::min(b, cap);
    S.occ.emplace(key, b);
  }
  if (cap > 0 && S.carve_for != smem) {
    // Fit the shared-memory carveout to b CTAs so the rest of the SM's
    // on-chip memory stays L1.
    int per_sm_smem = 0, reserved = 0;
    cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (per_sm_smem > 0) {
      const double need = (double)b * (double)(smem + (size_t)reserved);
      const int pct = std::min(100, (int)std::ceil(100.0 * need / per_sm_smem));
      cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    }
    S.carve_for = smem;
  }
  return b;
}

bits_status pool_alloc(void** p, size_t bytes, cudaStream_t st) {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  int dev = 0;
  BITS_CUDA_TRY(cudaGetDevice(&dev));
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
    if (!pools[dev]) {
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      BITS_CUDA_TRY(cudaMemPoolCreate(&pools[dev], &props));
      uint64_t keep = kPoolKeepBytes;
      BITS_CUDA_TRY(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    }
    pool = pools[dev];
  }
  BITS_CUDA_TRY(cudaMallocFromPoolAsync(p, bytes, pool, st));
  return BITS_OK;
}

bits_status cuda_status(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? BITS_ENOMEM : BITS_ECUDA;
}

bits_status read_device_error(const bits_db* db, cudaStream_t st, bool clear) {
  uint32_t h = 0;
  BITS_CUDA_TRY(cudaMemcpyAsync(&h, db->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  BITS_CUDA_TRY(cudaStreamSynchronize(st));
  if (clear && h) BITS_CUDA_TRY(cudaMemsetAsync(db->err, 0, sizeof(uint32_t), st));
  if (h & DEV_ERR_INTERNAL) {
    set_error("a device-side consistency check failed (index out of range); results are invalid");
    return BITS_EINTERNAL;
  }
  if (h & DEV_ERR_TIMEOUT) {
    set_error("a bounded device-side wait timed out; results are invalid");
    return BITS_ETIMEOUT;
  }
  if (h & DEV_ERR_INVALID) {
    set_error("an invalid interval was seen (query end < start, or outside its contig)");
    return BITS_EINVAL;
  }
  return BITS_OK;
}

// The sort of bits_build_db: starts into db->bs, ends into db->be (with
// the enumeration table's index sort when want_enum).  read_back = false:
// the keys-only sort runs without reading anything back (inputs checked).
bits_status sort_database(bits_db* db, const uint32_t* d_b, bool want_enum, cudaStream_t st,
                          bool read_back = true) {
  const uint32_t nn = db->n;
  if (nn) {
    RadixScratch ws{};
    const size_t sw = radix_status_words(nn);
    // With enumeration the sort carries indices: 4 more arrays of n words.
    const size_t words_n = align_up(sizeof(uint32_t) * nn, 256);
    const size_t scratch_bytes = (want_enum ? 6 : 2) * words_n +
                                 align_up(sizeof(uint32_t) * kRadixHistWords, 256) +
                                 align_up(sizeof(uint32_t) * sw * 8, 256) + 256;
    void* scratch = nullptr;
    const bits_status se = pool_alloc(&scratch, scratch_bytes, st);
    if (se != BITS_OK) return se;
    char* sb = static_cast<char*>(scratch);
    ws.tmp_s = reinterpret_cast<uint32_t*>(sb);
    sb += align_up(sizeof(uint32_t) * nn, 256);
    ws.tmp_e = reinterpret_cast<uint32_t*>(sb);
    sb += align_up(sizeof(uint32_t) * nn, 256);
    ws.hist = reinterpret_cast<uint32_t*>(sb);
    sb += align_up(sizeof(uint32_t) * kRadixHistWords, 256);
    ws.status = reinterpret_cast<uint32_t*>(sb);
    sb += align_up(sizeof(uint32_t) * sw * 8, 256);
    ws.tickets = reinterpret_cast<uint32_t*>(sb);
    sb += 256;
    bits_status s;
    if (want_enum) {
      SortSpec spec[2]{};
      uint32_t* idx_s = reinterpret_cast<uint32_t*>(sb);
      spec[0].comp = 0;
      spec[0].out_keys = db->bs;
      spec[0].tmp_keys = ws.tmp_s;
      spec[0].out_vals = idx_s;
      spec[0].tmp_vals = reinterpret_cast<uint32_t*>(sb + words_n);
      spec[1].comp = 1;
      spec[1].out_keys = db->be;
      spec[1].tmp_keys = ws.tmp_e;
      spec[1].out_vals = reinterpret_cast<uint32_t*>(sb + 2 * words_n);
      spec[1].tmp_vals = reinterpret_cast<uint32_t*>(sb + 3 * words_n);
      s = radix_sort_pairs(reinterpret_cast<const uint2*>(d_b), nn, spec, 0, db->err, ws, st,
                           nullptr);
      if (s == BITS_OK) s = launch_enum_gather(d_b, idx_s, nn, db->enum_e, st);
    } else {
      s = radix_sort_intervals(reinterpret_cast<const uint2*>(d_b), nn, db->bs, db->be, db->err,
                               ws, st, read_back);
    }
    pool_free(scratch, st);
    if (s != BITS_OK) return s;
  }
  return BITS_OK;
}

bits_status db_rebuild(bits_db* db, const uint32_t* d_b, cudaStream_t st) {
  if (db->has_rmi || db->enum_e) {
    set_error("db_rebuild: only plain databases are rebuilt in place");
    return BITS_EINVAL;
  }
  BITS_CUDA_TRY(cudaMemsetAsync(db->err, 0, sizeof(uint32_t), st));
  const bits_status s = sort_database(db, d_b, false, st, false);
  if (s != BITS_OK) return s;
  return build_levels(db, st);
}

}  // namespace bits

using namespace bits;

extern "C" {

const char* bits_last_error(void) { return g_last_error.c_str(); }

uint64_t bits_kernel_launches(void) { return g_launches.load(); }

bits_status bits_build_db(const uint32_t* d_b, uint64_t n, const bits_opts* opts, void* stream,
                          bits_db** out) {
  if (!out) {
    set_error("bits_build_db: out is NULL");
    return BITS_EINVAL;
  }
  *out = nullptr;
  if (n && !d_b) {
    set_error("bits_build_db: d_b is NULL");
    return BITS_EINVAL;
  }
  if (n >= (1ull << 30)) {
    set_error("bits_build_db: at most 2^30 - 1 database intervals are supported");
    return BITS_EOVERFLOW;
  }
  if (reinterpret_cast<uintptr_t>(d_b) % 8) {
    set_error("bits_build_db: d_b must be 8-byte aligned");
    return BITS_EINVAL;
  }
  bits_opts o{};
  if (opts) o = *opts;
  const int t = o.top_tree_log2 ? o.top_tree_log2 : 12;
  if (t < 2 || t > 14 || o.rmi_leaves_log2 < 0 || o.rmi_leaves_log2 > 22 ||
      (o.flags & ~BITS_FLAG_ENUMERATE) != 0 ||
      o.method < 0 || o.method > BITS_METHOD_MERGEPATH) {
    set_error("bits_build_db: option out of range");
    return BITS_EINVAL;
  }
  if (o.method == BITS_METHOD_RMI && o.rmi_leaves_log2 == 0) {
    set_error("bits_build_db: method RMI needs rmi_leaves_log2 > 0");
    return BITS_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t nn = (uint32_t)n;

  auto db = std::make_unique<bits_db>();
  BITS_CUDA_TRY(cudaGetDevice(&db->device));
  db->n = nn;
  plan_levels(nn, t, db->plan);
  db->method = o.method ? o.method : (o.rmi_leaves_log2 ? BITS_METHOD_AUTO : BITS_METHOD_SEARCH);
  db->has_rmi = o.rmi_leaves_log2 > 0;

  const bool want_enum = (o.flags & BITS_FLAG_ENUMERATE) != 0;
  // One allocation: bs | be | levels (both arrays) | top images | err | rmi leaves x 2
  // | enumeration pairs.
  const size_t n16 = std::max<uint32_t>(round16(nn), 16);
  const size_t off_bs = 0;
  const size_t off_be = align_up(off_bs + sizeof(uint32_t) * n16, 256);
  const size_t off_lv = align_up(off_be + sizeof(uint32_t) * n16, 256);
  const size_t off_top = align_up(off_lv + sizeof(uint32_t) * db->plan.level_words, 256);
  const size_t off_err = align_up(off_top + sizeof(uint32_t) * db->plan.top_words, 256);
  const size_t off_rmi = align_up(off_err + 256, 256);
  const size_t leaves = db->has_rmi ? (1ull << o.rmi_leaves_log2) : 0;
  const size_t off_enum = align_up(off_rmi + 2 * leaves * sizeof(bits_rmi_leaf), 256);
  const size_t total = off_enum + (want_enum ? sizeof(uint2) * std::max<uint32_t>(nn, 1) : 0);
  void* block = nullptr;
  {
    const bits_status as = pool_alloc(&block, total, st);
    if (as != BITS_OK) return as;
  }
  db->block = block;
  db->block_bytes = total;
  char* base = static_cast<char*>(block);
  db->bs = reinterpret_cast<uint32_t*>(base + off_bs);
  db->be = reinterpret_cast<uint32_t*>(base + off_be);
  db->levels = reinterpret_cast<uint32_t*>(base + off_lv);
  db->top = reinterpret_cast<uint32_t*>(base + off_top);
  db->err = reinterpret_cast<uint32_t*>(base + off_err);
  if (want_enum) db->enum_e = reinterpret_cast<uint2*>(base + off_enum);
  if (db->has_rmi) {
    db->rmi[0].leaves_log2 = db->rmi[1].leaves_log2 = o.rmi_leaves_log2;
    db->rmi[0].leaves = reinterpret_cast<bits_rmi_leaf*>(base + off_rmi);
    db->rmi[1].leaves = db->rmi[0].leaves + leaves;
  }
  auto fail = [&](bits_status s) {
    cudaStreamSynchronize(st);
    cudaFree(block);
    return s;
  };
  if (cudaMemsetAsync(db->err, 0, sizeof(uint32_t), st) != cudaSuccess)
    return fail(cuda_status(cudaGetLastError(), "cudaMemsetAsync"));

  {
    const bits_status s = sort_database(db.get(), d_b, want_enum, st);
    if (s != BITS_OK) return fail(s);
  }
  bits_status s = build_levels(db.get(), st);
  if (s != BITS_OK) return fail(s);
  if (db->has_rmi) {
    for (int a = 0; a < 2; ++a) {
      s = rmi_build(a ? db->be : db->bs, nn, db->rmi[a], st);
      if (s != BITS_OK) return fail(s);
    }
  }
  s = read_device_error(db.get(), st, false);
  if (s != BITS_OK) return fail(s);
  *out = db.release();
  return BITS_OK;
}

bits_status bits_count_method(const bits_db* db, int32_t method, const uint32_t* d_a, uint64_t n,
                              uint32_t* d_counts, uint64_t* d_total, void* stream) {
  if (!db || !d_total || (n && !d_a)) {
    set_error("bits_count: NULL argument");
    return BITS_EINVAL;
  }
  if (n >= (1ull << 32)) {
    set_error("bits_count: at most 2^32 - 1 queries per call");
    return BITS_EOVERFLOW;
  }
  if (reinterpret_cast<uintptr_t>(d_a) % 8 || reinterpret_cast<uintptr_t>(d_counts) % 4 ||
      reinterpret_cast<uintptr_t>(d_total) % 8) {
    set_error("bits_count: misaligned pointer (queries 8 B, counts 4 B, total 8 B)");
    return BITS_EINVAL;
  }
  if (method < BITS_METHOD_AUTO || method > BITS_METHOD_MERGEPATH) {
    set_error("bits_count: unknown method");
    return BITS_EINVAL;
  }
  if (method == BITS_METHOD_RMI && !db->has_rmi) {
    set_error("bits_count: database was built without a learned index");
    return BITS_ENOTIMPL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Method (for AUTO), shared-memory top and CTA size: pinned, tuned for
  // this size class (timed here the first time the class is seen), or the
  // defaults.
  TuneCount t;
  bits_status s = autotune_count(db, d_a, (uint32_t)n, d_counts, d_total, st, method, &t);
  if (s != BITS_OK) return s;
  return launch_count_tuned(db, t, d_a, (uint32_t)n, d_counts, d_total, st);
}

bits_status bits_count(const bits_db* db, const uint32_t* d_a, uint64_t n, uint32_t* d_counts,
                       uint64_t* d_total, void* stream) {
  if (!db) {
    set_error("bits_count: db is NULL");
    return BITS_EINVAL;
  }
  return bits_count_method(db, db->method, d_a, n, d_counts, d_total, stream);
}

bits_status bits_mc(const bits_db* db, int32_t method, const uint32_t* d_a, uint64_t n,
                    const uint32_t* d_contig_off, const uint32_t* d_contig_len, uint32_t n_contigs,
                    uint64_t seed, uint32_t shuffle_begin, uint32_t shuffle_end,
                    uint64_t* d_totals, uint64_t* h_observed, uint64_t* h_k_ge, double* h_pvalue,
                    void* stream) {
  if (!db || (n && !d_a) || !d_contig_off || !d_contig_len || n_contigs == 0 ||
      shuffle_end < shuffle_begin || (shuffle_end > shuffle_begin && !d_totals)) {
    set_error("bits_mc: bad argument");
    return BITS_EINVAL;
  }
  if (n >= (1ull << 32)) {
    set_error("bits_mc: at most 2^32 - 1 queries");
    return BITS_EOVERFLOW;
  }
  // The Monte-Carlo autotuner tunes the work-unit shape, not the method:
  // AUTO takes the plain search (faster than the learned index here).
  if (method == BITS_METHOD_AUTO) method = BITS_METHOD_SEARCH;
  if (method == BITS_METHOD_RMI && !db->has_rmi) {
    set_error("bits_mc: database was built without a learned index");
    return BITS_ENOTIMPL;
  }
  if (method != BITS_METHOD_SEARCH && method != BITS_METHOD_RMI) {
    set_error("bits_mc: method must be SEARCH or RMI");
    return BITS_EINVAL;
  }
  return run_mc(const_cast<bits_db*>(db), method, d_a, (uint32_t)n, d_contig_off, d_contig_len,
                n_contigs, seed, shuffle_begin, shuffle_end, d_totals, h_observed, h_k_ge,
                h_pvalue, static_cast<cudaStream_t>(stream));
}

bits_status bits_count_matrix(const bits_db* const* dbs, uint32_t n_db,
                              const uint32_t* const* d_as, const uint64_t* n_as, uint32_t n_sets,
                              uint64_t* d_matrix, void* stream) {
  if ((n_db && !dbs) || (n_sets && (!d_as || !n_as)) || (n_db && n_sets && !d_matrix)) {
    set_error("bits_count_matrix: NULL argument");
    return BITS_EINVAL;
  }
  for (uint32_t j = 0; j < n_db; ++j)
    if (!dbs[j]) {
      set_error("bits_count_matrix: NULL database handle");
      return BITS_EINVAL;
    }
  for (uint32_t i = 0; i < n_sets; ++i) {
    if (n_as[i] >= (1ull << 32)) {
      set_error("bits_count_matrix: a query set has 2^32 or more intervals");
      return BITS_EOVERFLOW;
    }
    if (n_as[i] && (!d_as[i] || reinterpret_cast<uintptr_t>(d_as[i]) % 8)) {
      set_error("bits_count_matrix: query set pointer NULL or not 8-byte aligned");
      return BITS_EINVAL;
    }
  }
  return run_count_matrix(dbs, n_db, d_as, n_as, n_sets, d_matrix,
                          static_cast<cudaStream_t>(stream));
}

bits_status bits_count_matrix_db(const bits_db* const* a_dbs, uint32_t n_a,
                                 const bits_db* const* b_dbs, uint32_t n_b, uint64_t* d_matrix,
                                 void* stream) {
  if ((n_a && !a_dbs) || (n_b && !b_dbs) || (n_a && n_b && !d_matrix)) {
    set_error("bits_count_matrix_db: NULL argument");
    return BITS_EINVAL;
  }
  for (uint32_t i = 0; i < n_a; ++i)
    if (!a_dbs[i]) {
      set_error("bits_count_matrix_db: NULL database handle");
      return BITS_EINVAL;
    }
  for (uint32_t j = 0; j < n_b; ++j)
    if (!b_dbs[j]) {
      set_error("bits_count_matrix_db: NULL database handle");
      return BITS_EINVAL;
    }
  return run_count_matrix_db(a_dbs, n_a, b_dbs, n_b, d_matrix, static_cast<cudaStream_t>(stream));
}

bits_status bits_enumerate_offsets(const bits_db* db, const uint32_t* d_a, uint64_t n,
                                   uint64_t* d_offsets, void* stream) {
  if (!db || !d_offsets || (n && !d_a)) {
    set_error("bits_enumerate_offsets: NULL argument");
    return BITS_EINVAL;
  }
  if (n >= (1ull << 32)) {
    set_error("bits_enumerate_offsets: n must be below 2^32");
    return BITS_EOVERFLOW;
  }
  if ((reinterpret_cast<uintptr_t>(d_a) | reinterpret_cast<uintptr_t>(d_offsets)) & 7u) {
    set_error("bits_enumerate_offsets: pointers must be 8-byte aligned");
    return BITS_EINVAL;
  }
  return run_enumerate_offsets(db, d_a, (uint32_t)n, d_offsets, static_cast<cudaStream_t>(stream));
}

bits_status bits_enumerate_pairs(const bits_db* db, const uint32_t* d_a, uint64_t n,
                                 const uint64_t* d_offsets, uint32_t* d_pairs, void* stream) {
  if (!db || !d_offsets || (n && !d_a)) {
    set_error("bits_enumerate_pairs: NULL argument");
    return BITS_EINVAL;
  }
  if (!db->enum_e) {
    set_error("bits_enumerate_pairs: database built without BITS_FLAG_ENUMERATE");
    return BITS_ENOTIMPL;
  }
  if (n >= (1ull << 32)) {
    set_error("bits_enumerate_pairs: n must be below 2^32");
    return BITS_EOVERFLOW;
  }
  if ((reinterpret_cast<uintptr_t>(d_a) | reinterpret_cast<uintptr_t>(d_offsets) |
       reinterpret_cast<uintptr_t>(d_pairs)) & 7u) {
    set_error("bits_enumerate_pairs: pointers must be 8-byte aligned");
    return BITS_EINVAL;
  }
  return run_enumerate_pairs(db, d_a, (uint32_t)n, d_offsets, d_pairs,
                             static_cast<cudaStream_t>(stream));
}

bits_status bits_mc_matrix(const bits_db* const* dbs, uint32_t n_db, const uint32_t* const* d_as,
                           const uint64_t* n_as, uint32_t n_sets, const uint32_t* d_contig_off,
                           const uint32_t* d_contig_len, uint32_t n_contigs, uint64_t seed,
                           uint32_t shuffle_begin, uint32_t shuffle_end, uint64_t* d_observed,
                           uint64_t* d_totals, bits_mc_stat* d_stats, void* stream) {
  if ((n_db && !dbs) || (n_sets && (!d_as || !n_as)) || shuffle_end < shuffle_begin) {
    set_error("bits_mc_matrix: NULL argument or shuffle_end < shuffle_begin");
    return BITS_EINVAL;
  }
  if (n_db == 0 || n_sets == 0) return BITS_OK;
  if (!d_observed || (shuffle_end > shuffle_begin && !d_totals) || !d_contig_off ||
      !d_contig_len || n_contigs == 0) {
    set_error("bits_mc_matrix: NULL output or empty contig table");
    return BITS_EINVAL;
  }
  if (n_contigs > 4096) {
    set_error("bits_mc_matrix: at most 4096 contigs");
    return BITS_EOVERFLOW;
  }
  if ((reinterpret_cast<uintptr_t>(d_observed) | reinterpret_cast<uintptr_t>(d_totals) |
       reinterpret_cast<uintptr_t>(d_stats)) & 7u) {
    set_error("bits_mc_matrix: outputs must be 8-byte aligned");
    return BITS_EINVAL;
  }
  for (uint32_t j = 0; j < n_db; ++j)
    if (!dbs[j]) {
      set_error("bits_mc_matrix: NULL database handle");
      return BITS_EINVAL;
    }
  for (uint32_t i = 0; i < n_sets; ++i) {
    if (n_as[i] >= (1ull << 32)) {
      set_error("bits_mc_matrix: a query set has 2^32 or more intervals");
      return BITS_EOVERFLOW;
    }
    if (n_as[i] && (!d_as[i] || reinterpret_cast<uintptr_t>(d_as[i]) % 8)) {
      set_error("bits_mc_matrix: query set pointer NULL or not 8-byte aligned");
      return BITS_EINVAL;
    }
  }
  return run_mc_matrix(dbs, n_db, d_as, n_as, n_sets, d_contig_off, d_contig_len, n_contigs, seed,
                       shuffle_begin, shuffle_end, d_observed, d_totals, d_stats,
                       static_cast<cudaStream_t>(stream));
}

bits_status bits_mc_summary(const uint64_t* d_totals, uint32_t n_shuffles, uint32_t n_tests,
                            const uint64_t* d_observed, bits_mc_stat* d_stats, void* stream) {
  if (n_tests == 0) return BITS_OK;
  if (!d_observed || !d_stats || (n_shuffles && !d_totals)) {
    set_error("bits_mc_summary: NULL argument");
    return BITS_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(d_totals) | reinterpret_cast<uintptr_t>(d_observed) |
       reinterpret_cast<uintptr_t>(d_stats)) & 7u) {
    set_error("bits_mc_summary: pointers must be 8-byte aligned");
    return BITS_EINVAL;
  }
  return launch_mc_summary(d_totals, n_shuffles, n_tests, d_observed, d_stats,
                           static_cast<cudaStream_t>(stream));
}

bits_status bits_project(const uint32_t* d_contig, const uint32_t* d_start, const uint32_t* d_end,
                         uint64_t n, const uint32_t* d_contig_off, const uint32_t* d_contig_len,
                         uint32_t n_contigs, int32_t closed, uint32_t* d_out,
                         uint64_t* d_n_rejected, void* stream) {
  if (n >= (1ull << 32)) {
    set_error("bits_project: n must be below 2^32");
    return BITS_EOVERFLOW;
  }
  if (closed != 0 && closed != 1) {
    set_error("bits_project: closed must be 0 or 1");
    return BITS_EINVAL;
  }
  if (n && (!d_start || !d_end || !d_out || (n_contigs && !d_contig))) {
    set_error("bits_project: NULL interval array");
    return BITS_EINVAL;
  }
  if (n_contigs && (!d_contig_off || !d_contig_len)) {
    set_error("bits_project: NULL contig table");
    return BITS_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(d_out) & 7u) || (reinterpret_cast<uintptr_t>(d_start) & 3u) ||
      (reinterpret_cast<uintptr_t>(d_end) & 3u) || (reinterpret_cast<uintptr_t>(d_contig) & 3u)) {
    set_error("bits_project: misaligned pointer (out needs 8 bytes, inputs 4)");
    return BITS_EINVAL;
  }
  return launch_project(d_contig, d_start, d_end, n, d_contig_off, d_contig_len, n_contigs,
                        closed != 0, d_out, d_n_rejected, static_cast<cudaStream_t>(stream));
}

bits_status bits_db_info(const bits_db* db, const uint32_t** d_bs, const uint32_t** d_be,
                         uint64_t* n, int32_t* has_rmi) {
  if (!db) {
    set_error("bits_db_info: db is NULL");
    return BITS_EINVAL;
  }
  if (d_bs) *d_bs = db->bs;
  if (d_be) *d_be = db->be;
  if (n) *n = db->n;
  if (has_rmi) *has_rmi = db->has_rmi ? 1 : 0;
  return BITS_OK;
}

bits_status bits_db_rmi(const bits_db* db, int32_t which, const void** d_leaves,
                        uint32_t* n_leaves, float* root_slope, float* root_icpt) {
  if (!db || which < 0 || which > 1) {
    set_error("bits_db_rmi: bad argument");
    return BITS_EINVAL;
  }
  if (!db->has_rmi) {
    set_error("bits_db_rmi: database was built without a learned index");
    return BITS_ENOTIMPL;
  }
  const bits_rmi& r = db->rmi[which];
  if (d_leaves) *d_leaves = r.leaves;
  if (n_leaves) *n_leaves = 1u << r.leaves_log2;
  if (root_slope) *root_slope = r.root_slope;
  if (root_icpt) *root_icpt = r.root_icpt;
  return BITS_OK;
}

bits_status bits_check(const bits_db* db, void* stream) {
  if (!db) {
    set_error("bits_check: db is NULL");
    return BITS_EINVAL;
  }
  return read_device_error(db, static_cast<cudaStream_t>(stream), true);
}

void bits_free(bits_db* db) {
  if (!db) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != db->device) cudaSetDevice(db->device);
  release_mc_graphs(db);
  release_matrix_graphs(db);
  release_mc_matrix_graphs(db);
  // The block comes from the stream-ordered pool, and cudaFree does not wait
  // for such memory: finish every stream's work on the device first.
  cudaDeviceSynchronize();
  cudaFree(db->block);
  if (prev != db->device) cudaSetDevice(prev);
  delete db;
}

}  // extern "C"
