// All-pairs count matrix (the screen of Sec. "Novel genomic relationships"):
// M[i][j] = total(A_i, B_j) for every query set A_i and database B_j, in one
// persistent launch.
//
// bits_count_matrix takes the query sets as (start, end) pairs.  Work is
// split by query count: a unit is (database j, query set i, chunk of up to C
// queries; C = 8192 by default, tuned per argument shape among 4096 .. 32768
// by timing the launch once per candidate on the first call), and units are
// listed database by database, largest database first, so the deepest
// (slowest) searches start early and the small units fill the tail.  CTAs
// take units from an atomic ticket; a CTA reloads its shared-memory top
// level only when its unit's database differs from the previous one.  Each
// unit reduces its chunk to one uint64 and adds it to its matrix entry with
// one atomic.  Per database the search method (plain 16-ary tree or learned
// index) comes from the autotuner, timed on a sample of the queries the
// first time a size class is seen.
//
// bits_count_matrix_db takes the query sets as databases too (every track of
// the screen is both a query set and a database).  Summing Algorithm 2's
// ICount over A needs only A's keys, each array on its own:
//     total(A, B) = sum_{x in A_E} #(B_S < x) - sum_{x in A_S} #(B_E <= x),
// and counting the same pairs from B's side gives
//     total(A, B) = sum_{x in B_E} #(A_S < x) - sum_{x in B_S} #(A_E <= x).
// So each pair is counted from the sorted arrays of its smaller side,
// searched in the larger side's tree: the k-th sorted start and k-th sorted
// end of the smaller side form one search pair (x_S, x_E), and its ICount
// against the larger side is #(T_S < x_E) - #(T_E < x_S + 1), exactly a
// query's.  A pair then costs min(|A|, |B|) searches instead of |A|, and the
// keys arrive sorted, so neighbouring searches share tree nodes in L1 and
// L2.  Units are as above with the larger side as the database.
//
// Each call (zero M, reset the ticket, the persistent launch) is captured
// once per argument set into a CUDA graph and replayed.
#include <algorithm>
#include <functional>
#include <memory>
#include <vector>

#include "allpairs.cuh"
#include "count.cuh"
#include "rmi.cuh"
#include "rmi_search.cuh"
#include "search.cuh"
#include "tune.cuh"

namespace bits {
namespace {

constexpr int kApBlock = 256;

struct MatDb {
  LevelIndex L;
  RmiView R;
  uint32_t nb;
  int method;
  uint32_t* err;
};

// `count` search pairs from `start` of key source `set`, searched in
// database `db`; the total goes to matrix entry `out`.
struct MatUnit {
  uint32_t db, set, start, count, out;
};

struct MatArgs {
  const MatDb* dbs;
  const MatUnit* units;
  uint32_t n_units;
  const uint2* const* sets;     // bits_count_matrix: the query sets' (start, end) pairs
  const uint32_t* const* keys;  // bits_count_matrix_db: [2k] sorted starts, [2k + 1] sorted ends
  unsigned long long* matrix;
  uint32_t* ticket;
};

template <bool kSorted>
__global__ void __launch_bounds__(kApBlock)
k_allpairs(MatArgs P) {
  extern __shared__ __align__(16) uint32_t s_top[];
  __shared__ MatDb s_db;
  __shared__ uint32_t s_unit;
  __shared__ int s_cur;
  __shared__ unsigned long long s_red[32];
  if (threadIdx.x == 0) s_cur = -1;
  for (;;) {
    if (threadIdx.x == 0) s_unit = atomicAdd(P.ticket, 1u);
    __syncthreads();
    const uint32_t u = s_unit;
    if (u >= P.n_units) break;
    const MatUnit U = P.units[u];
    if ((int)U.db != s_cur) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(P.dbs + U.db);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&s_db);
      for (uint32_t k = threadIdx.x; k < sizeof(MatDb) / 4; k += blockDim.x) dst[k] = src[k];
      __syncthreads();
      if (s_db.method != BITS_METHOD_RMI) load_top(s_top, s_db.L);
      if (threadIdx.x == 0) s_cur = (int)U.db;
      __syncthreads();
    }
    const uint2* A = kSorted ? nullptr : P.sets[U.set] + U.start;
    const uint32_t* XS = kSorted ? P.keys[2 * U.set] + U.start : nullptr;
    const uint32_t* XE = kSorted ? P.keys[2 * U.set + 1] + U.start : nullptr;
    const bool rmi = s_db.method == BITS_METHOD_RMI;
    const uint32_t nb = s_db.nb;
    unsigned long long acc = 0ull;
    bool bad = false;
    for (uint32_t base = 0; base < U.count; base += kApBlock) {
      const uint32_t i = base + threadIdx.x;
      const bool valid = i < U.count;
      uint2 q = make_uint2(0u, 0u);
      if (valid) q = kSorted ? make_uint2(__ldg(XS + i), __ldg(XE + i)) : __ldg(A + i);
      const uint32_t key_s = q.y, key_e = q.x + 1u;
      uint32_t rs, re;
      if (rmi) {
        rmi_rank2(s_db.R, s_db.L, nb, key_s, key_e, rs, re);
      } else {
        top_rank2(s_top, s_db.L.top_size, key_s, key_e, rs, re);
        quad_descend(s_db.L, rs, key_s, re, key_e);
      }
      uint32_t c = icount_from_ranks(rs, re, q.x, nb);
      if (q.y < q.x) {  // an inverted query (never a pair of sorted database keys)
        c = 0u;
        bad = true;
      }
      if (valid) acc += c;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_dev_error(s_db.err, DEV_ERR_INVALID);
    const unsigned long long sum = block_sum_u64(acc, s_red);
    if (threadIdx.x == 0 && sum) atomicAdd(P.matrix + U.out, sum);
    __syncthreads();
  }
}

template <bool kSorted>
int ap_blocks_per_sm(size_t smem) {
  return kernel_blocks_per_sm(reinterpret_cast<const void*>(k_allpairs<kSorted>), kApBlock, smem);
}

struct MatGraph {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  void* dev = nullptr;  // descriptors | units | source pointers | ticket
  uint64_t kernels = 0;
  ~MatGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (dev) cudaFree(dev);
  }
};

// At most 16 argument sets keep a captured graph (graph_cache.cuh).
GraphCache<std::vector<uint64_t>, MatGraph> g_graphs(16);

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Builds g: device copies of the descriptors, the unit list and the source
// pointers; the chunk size (tuned here on the first call of an argument
// shape unless pinned or recorded: one timed launch per candidate after a
// warm-up round); and the captured graph of the whole call.
template <bool kSorted>
bits_status build_matrix_graph(MatGraph& g, const std::vector<MatDb>& hd,
                               const std::vector<const void*>& sources, size_t max_top,
                               const std::function<std::vector<MatUnit>(uint32_t)>& make_units,
                               const char* tune_kind, uint64_t total_q, uint64_t total_db,
                               uint32_t n_sets, uint64_t* d_matrix, size_t n_out,
                               cudaStream_t st) {
  const uint32_t n_db = (uint32_t)hd.size();
  bool tuned = false;
  uint32_t chunk =
      (uint32_t)ap_chunk_params(total_q, total_db, n_db, n_sets, &tuned, tune_kind);
  // Room for the unit list of the smallest candidate chunk.
  const size_t max_units = std::max<size_t>(make_units(kApChunks[0]).size(), 1);
  const size_t off_units = align256(sizeof(MatDb) * n_db);
  const size_t off_src = off_units + align256(sizeof(MatUnit) * max_units);
  const size_t off_ticket = off_src + align256(sizeof(void*) * std::max<size_t>(sources.size(), 1));
  BITS_CUDA_TRY(cudaMalloc(&g.dev, off_ticket + 256));
  char* base = static_cast<char*>(g.dev);
  BITS_CUDA_TRY(cudaMemcpy(base, hd.data(), sizeof(MatDb) * n_db, cudaMemcpyHostToDevice));
  if (!sources.empty())
    BITS_CUDA_TRY(cudaMemcpy(base + off_src, sources.data(), sizeof(void*) * sources.size(),
                             cudaMemcpyHostToDevice));
  MatArgs P{};
  P.dbs = reinterpret_cast<const MatDb*>(base);
  P.units = reinterpret_cast<const MatUnit*>(base + off_units);
  if (kSorted) P.keys = reinterpret_cast<const uint32_t* const*>(base + off_src);
  else P.sets = reinterpret_cast<const uint2* const*>(base + off_src);
  P.matrix = reinterpret_cast<unsigned long long*>(d_matrix);
  P.ticket = reinterpret_cast<uint32_t*>(base + off_ticket);
  const size_t smem = sizeof(uint32_t) * 2 * max_top;
  const uint32_t per_sm_grid = (uint32_t)(ap_blocks_per_sm<kSorted>(smem) * sm_count());
  auto upload = [&](uint32_t c) -> bits_status {
    const std::vector<MatUnit> units = make_units(c);
    if (!units.empty())
      BITS_CUDA_TRY(cudaMemcpy(base + off_units, units.data(), sizeof(MatUnit) * units.size(),
                               cudaMemcpyHostToDevice));
    P.n_units = (uint32_t)units.size();
    return BITS_OK;
  };
  if (!tuned && !stream_capturing(st)) {
    cudaEvent_t e0, e1;
    BITS_CUDA_TRY(cudaEventCreate(&e0));
    BITS_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    uint32_t best_c = chunk;
    bits_status s = BITS_OK;
    for (int round = 0; round < 2 && s == BITS_OK; ++round)
      for (int c : kApChunks) {
        s = upload((uint32_t)c);
        if (s != BITS_OK) break;
        const uint32_t grid = std::min<uint32_t>(std::max<uint32_t>(P.n_units, 1), per_sm_grid);
        cudaMemsetAsync(d_matrix, 0, sizeof(uint64_t) * n_out, st);
        cudaMemsetAsync(P.ticket, 0, sizeof(uint32_t), st);
        cudaEventRecord(e0, st);
        k_allpairs<kSorted><<<grid, kApBlock, smem, st>>>(P);
        count_launch();
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          s = cuda_status(cudaGetLastError(), "count_matrix tuning");
          break;
        }
        if (round > 0 && ms < best) {
          best = ms;
          best_c = (uint32_t)c;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != BITS_OK) return s;
    chunk = best_c;
    ap_chunk_record(total_q, total_db, n_db, n_sets, (int)chunk, tune_kind);
  }
  {
    const bits_status s = upload(chunk);
    if (s != BITS_OK) return s;
  }
  const uint32_t grid = std::min<uint32_t>(std::max<uint32_t>(P.n_units, 1), per_sm_grid);

  cudaStream_t cap = nullptr;
  BITS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cap);
    return cuda_status(e, "cudaStreamBeginCapture");
  }
  cudaMemsetAsync(d_matrix, 0, sizeof(uint64_t) * n_out, cap);
  cudaMemsetAsync(P.ticket, 0, sizeof(uint32_t), cap);
  k_allpairs<kSorted><<<grid, kApBlock, smem, cap>>>(P);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cap, &graph);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture(count_matrix)");
  g.graph = graph;
  BITS_CUDA_TRY(cudaGraphInstantiate(&g.exec, graph, 0));
  g.kernels = 1;
  return BITS_OK;
}

bits_status launch_graph(const std::shared_ptr<MatGraph>& g, cudaStream_t st) {
  BITS_CUDA_TRY(cudaGraphLaunch(g->exec, st));
  count_launch((uint32_t)g->kernels);
  return BITS_OK;
}

MatDb plain_descriptor(const bits_db* db) {
  MatDb d{};
  d.L = db->lvl;
  d.R = RmiView{};
  d.nb = db->n;
  d.method = BITS_METHOD_SEARCH;
  d.err = db->err;
  return d;
}

}  // namespace

bits_status run_count_matrix(const bits_db* const* dbs, uint32_t n_db,
                             const uint32_t* const* d_as, const uint64_t* n_as, uint32_t n_sets,
                             uint64_t* d_matrix, cudaStream_t st) {
  if (n_db == 0 || n_sets == 0) return BITS_OK;
  std::vector<uint64_t> key;
  key.push_back(reinterpret_cast<uintptr_t>(d_matrix) ^ ((uint64_t)pinned_tuning().ap_chunk << 48));
  for (uint32_t j = 0; j < n_db; ++j) key.push_back(reinterpret_cast<uintptr_t>(dbs[j]));
  for (uint32_t i = 0; i < n_sets; ++i) {
    key.push_back(reinterpret_cast<uintptr_t>(d_as[i]));
    key.push_back(n_as[i]);
  }
  std::shared_ptr<MatGraph> g = g_graphs.find(key);
  if (!g) {
    // Search method per database: the autotuner, timed on a sample of the
    // largest query set (at most 2^16 queries).
    uint32_t big = 0;
    for (uint32_t i = 1; i < n_sets; ++i)
      if (n_as[i] > n_as[big]) big = i;
    const uint32_t n_sample = (uint32_t)std::min<uint64_t>(n_as[big], 1u << 16);
    std::vector<MatDb> hd(n_db);
    uint64_t* d_tmp = nullptr;
    {
      const bits_status as = pool_alloc(reinterpret_cast<void**>(&d_tmp), sizeof(uint64_t), st);
      if (as != BITS_OK) return as;
    }
    size_t max_top = 4;
    for (uint32_t j = 0; j < n_db; ++j) {
      int m = BITS_METHOD_SEARCH;
      if (dbs[j]->has_rmi && n_sample) {
        TuneCount t;
        bits_status s = autotune_count(dbs[j], d_as[big], n_sample, nullptr, d_tmp, st,
                                       BITS_METHOD_AUTO, &t);
        if (s != BITS_OK) {
          pool_free(d_tmp, st);
          return s;
        }
        m = t.method;
      }
      hd[j] = plain_descriptor(dbs[j]);
      hd[j].R = dbs[j]->has_rmi ? rmi_view(dbs[j]) : RmiView{};
      hd[j].method = m;
      if (m != BITS_METHOD_RMI) max_top = std::max<size_t>(max_top, top_words(dbs[j]->lvl.top_size));
    }
    pool_free(d_tmp, st);
    // Units: largest database first, then set by set, `chunk` queries each.
    std::vector<uint32_t> order(n_db);
    for (uint32_t j = 0; j < n_db; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t x, uint32_t y) { return dbs[x]->n > dbs[y]->n; });
    auto make_units = [&](uint32_t chunk) {
      std::vector<MatUnit> units;
      for (uint32_t j : order)
        for (uint32_t i = 0; i < n_sets; ++i)
          for (uint64_t s0 = 0; s0 < n_as[i]; s0 += chunk)
            units.push_back(MatUnit{j, i, (uint32_t)s0,
                                    (uint32_t)std::min<uint64_t>(chunk, n_as[i] - s0),
                                    i * n_db + j});
      return units;
    };
    uint64_t total_q = 0, total_db = 0;
    for (uint32_t i = 0; i < n_sets; ++i) total_q += n_as[i];
    for (uint32_t j = 0; j < n_db; ++j) total_db += dbs[j]->n;
    std::vector<const void*> sets(d_as, d_as + n_sets);
    g = std::make_shared<MatGraph>();
    const bits_status s =
        build_matrix_graph<false>(*g, hd, sets, max_top, make_units, "allpairs", total_q, total_db,
                                  n_sets, d_matrix, (size_t)n_sets * n_db, st);
    if (s != BITS_OK) return s;
    g_graphs.put(key, g);
  }
  return launch_graph(g, st);
}

bits_status run_count_matrix_db(const bits_db* const* a_dbs, uint32_t n_a,
                                const bits_db* const* b_dbs, uint32_t n_b, uint64_t* d_matrix,
                                cudaStream_t st) {
  if (n_a == 0 || n_b == 0) return BITS_OK;
  // Key tag 1 keeps these graphs apart from bits_count_matrix's.
  std::vector<uint64_t> key;
  key.push_back(reinterpret_cast<uintptr_t>(d_matrix) ^ ((uint64_t)pinned_tuning().ap_chunk << 48) ^
                (1ull << 47));
  for (uint32_t i = 0; i < n_a; ++i) key.push_back(reinterpret_cast<uintptr_t>(a_dbs[i]));
  key.push_back(0);  // separates the two lists
  for (uint32_t j = 0; j < n_b; ++j) key.push_back(reinterpret_cast<uintptr_t>(b_dbs[j]));
  std::shared_ptr<MatGraph> g = g_graphs.find(key);
  if (!g) {
    // Databases 0 .. n_a - 1 are the A sets, n_a .. n_a + n_b - 1 the B sets;
    // each is searched with the plain tree, and each is a key source through
    // its sorted arrays.
    const uint32_t n_all = n_a + n_b;
    std::vector<const bits_db*> all(a_dbs, a_dbs + n_a);
    all.insert(all.end(), b_dbs, b_dbs + n_b);
    std::vector<MatDb> hd(n_all);
    std::vector<const void*> keys(2 * (size_t)n_all);
    size_t max_top = 4;
    for (uint32_t k = 0; k < n_all; ++k) {
      hd[k] = plain_descriptor(all[k]);
      keys[2 * k] = all[k]->bs;
      keys[2 * k + 1] = all[k]->be;
      max_top = std::max<size_t>(max_top, top_words(all[k]->lvl.top_size));
    }
    // Pair (i, j): keys from its smaller side, the tree of its larger side
    // (A_i on a tie).
    struct Pair {
      uint32_t tree, src, n, out;
    };
    std::vector<Pair> pairs;
    uint64_t total_keys = 0;
    for (uint32_t i = 0; i < n_a; ++i)
      for (uint32_t j = 0; j < n_b; ++j) {
        const bool a_keys = a_dbs[i]->n <= b_dbs[j]->n;
        const Pair p{a_keys ? n_a + j : i, a_keys ? i : n_a + j,
                     a_keys ? a_dbs[i]->n : b_dbs[j]->n, i * n_b + j};
        total_keys += p.n;
        if (p.n) pairs.push_back(p);
      }
    // Units: largest tree first (deepest searches start early), `chunk` keys each.
    std::stable_sort(pairs.begin(), pairs.end(), [&](const Pair& x, const Pair& y) {
      return all[x.tree]->n > all[y.tree]->n ||
             (all[x.tree]->n == all[y.tree]->n && x.tree < y.tree);
    });
    auto make_units = [&](uint32_t chunk) {
      std::vector<MatUnit> units;
      for (const Pair& p : pairs)
        for (uint32_t s0 = 0; s0 < p.n; s0 += chunk)
          units.push_back(MatUnit{p.tree, p.src, s0, std::min<uint32_t>(chunk, p.n - s0), p.out});
      return units;
    };
    uint64_t total_db = 0;
    for (uint32_t k = 0; k < n_all; ++k) total_db += all[k]->n;
    g = std::make_shared<MatGraph>();
    const bits_status s = build_matrix_graph<true>(*g, hd, keys, max_top, make_units,
                                                   "allpairs_db", total_keys, total_db, n_a, d_matrix,
                                                   (size_t)n_a * n_b, st);
    if (s != BITS_OK) return s;
    g_graphs.put(key, g);
  }
  return launch_graph(g, st);
}

void release_matrix_graphs(const bits_db* db) {
  g_graphs.erase_if([db](const std::vector<uint64_t>& key) {
    for (size_t k = 1; k < key.size(); ++k)
      if (key[k] == reinterpret_cast<uintptr_t>(db)) return true;
    return false;
  });
}

}  // namespace bits
