// All-pairs count matrix (the screen of Sec. "Novel genomic relationships"):
// M[i][j] = total(A_i, B_j) for every query set A_i and database B_j, in one
// persistent launch.
//
// Work is split by query count: a unit is (database j, query set i, chunk of
// up to C queries; C = 8192 by default, tuned per argument shape among 4096
// .. 32768 by timing the launch once per candidate on the first call), and
// units are listed database by database, largest
// database first, so the deepest (slowest) searches start early and the
// small units fill the tail.  CTAs take units from an atomic ticket; a CTA
// reloads its shared-memory top level only when its unit's database differs
// from the previous one.  Each unit reduces its chunk to one uint64 and adds
// it to M[i][j] with one atomic.
//
// Per database the search method (plain 16-ary tree or learned index) comes
// from the autotuner, timed on a sample of the queries the first time a size
// class is seen.  The whole call (zero M, reset the ticket, the persistent
// launch) is captured once per argument set into a CUDA graph and replayed.
#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
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

struct MatUnit {
  uint32_t db, set, start, count;
};

struct MatArgs {
  const MatDb* dbs;
  const MatUnit* units;
  uint32_t n_units;
  const uint2* const* sets;
  unsigned long long* matrix;
  uint32_t n_db;
  uint32_t* ticket;
};

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
    const uint2* A = P.sets[U.set] + U.start;
    const bool rmi = s_db.method == BITS_METHOD_RMI;
    const uint32_t nb = s_db.nb;
    unsigned long long acc = 0ull;
    bool bad = false;
    for (uint32_t base = 0; base < U.count; base += kApBlock) {
      const uint32_t i = base + threadIdx.x;
      const bool valid = i < U.count;
      uint2 q = make_uint2(0u, 0u);
      if (valid) q = __ldg(A + i);
      const uint32_t key_s = q.y, key_e = q.x + 1u;
      uint32_t rs, re;
      if (rmi) {
        rmi_rank2(s_db.R, s_db.L, nb, key_s, key_e, rs, re);
      } else {
        top_rank2(s_top, s_db.L.top_size, key_s, key_e, rs, re);
        quad_descend(s_db.L, rs, key_s, re, key_e);
      }
      uint32_t c = icount_from_ranks(rs, re, q.x, nb);
      if (q.y < q.x) {
        c = 0u;
        bad = true;
      }
      if (valid) acc += c;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_dev_error(s_db.err, DEV_ERR_INVALID);
    const unsigned long long sum = block_sum_u64(acc, s_red);
    if (threadIdx.x == 0 && sum) atomicAdd(P.matrix + (size_t)U.set * P.n_db + U.db, sum);
    __syncthreads();
  }
}

int ap_blocks_per_sm(size_t smem) {
  return kernel_blocks_per_sm(reinterpret_cast<const void*>(k_allpairs), kApBlock, smem);
}

struct MatGraph {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  void* dev = nullptr;  // descriptors | units | set pointers | ticket
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
      hd[j].L = dbs[j]->lvl;
      hd[j].R = dbs[j]->has_rmi ? rmi_view(dbs[j]) : RmiView{};
      hd[j].nb = dbs[j]->n;
      hd[j].method = m;
      hd[j].err = dbs[j]->err;
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
                                    (uint32_t)std::min<uint64_t>(chunk, n_as[i] - s0)});
      return units;
    };
    uint64_t total_q = 0, total_db = 0;
    for (uint32_t i = 0; i < n_sets; ++i) total_q += n_as[i];
    for (uint32_t j = 0; j < n_db; ++j) total_db += dbs[j]->n;
    bool tuned = false;
    uint32_t chunk = (uint32_t)ap_chunk_params(total_q, total_db, n_db, n_sets, &tuned);
    // Room for the unit list of the smallest candidate chunk.
    const size_t max_units = std::max<size_t>(make_units(kApChunks[0]).size(), 1);
    g = std::make_shared<MatGraph>();
    const size_t off_units = align256(sizeof(MatDb) * n_db);
    const size_t off_sets = off_units + align256(sizeof(MatUnit) * max_units);
    const size_t off_ticket = off_sets + align256(sizeof(void*) * n_sets);
    BITS_CUDA_TRY(cudaMalloc(&g->dev, off_ticket + 256));
    char* base = static_cast<char*>(g->dev);
    std::vector<const void*> sets(d_as, d_as + n_sets);
    BITS_CUDA_TRY(cudaMemcpy(base, hd.data(), sizeof(MatDb) * n_db, cudaMemcpyHostToDevice));
    BITS_CUDA_TRY(cudaMemcpy(base + off_sets, sets.data(), sizeof(void*) * n_sets,
                             cudaMemcpyHostToDevice));
    MatArgs P{};
    P.dbs = reinterpret_cast<const MatDb*>(base);
    P.units = reinterpret_cast<const MatUnit*>(base + off_units);
    P.sets = reinterpret_cast<const uint2* const*>(base + off_sets);
    P.matrix = reinterpret_cast<unsigned long long*>(d_matrix);
    P.n_db = n_db;
    P.ticket = reinterpret_cast<uint32_t*>(base + off_ticket);
    const size_t smem = sizeof(uint32_t) * 2 * max_top;
    const uint32_t per_sm_grid = (uint32_t)(ap_blocks_per_sm(smem) * sm_count());
    auto upload = [&](uint32_t c) -> bits_status {
      const std::vector<MatUnit> units = make_units(c);
      if (!units.empty())
        BITS_CUDA_TRY(cudaMemcpy(base + off_units, units.data(), sizeof(MatUnit) * units.size(),
                                 cudaMemcpyHostToDevice));
      P.n_units = (uint32_t)units.size();
      return BITS_OK;
    };
    if (!tuned && !stream_capturing(st)) {
      // Time one launch per candidate chunk (after a warm-up launch of each)
      // and record the fastest for this argument shape.
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
          cudaMemsetAsync(d_matrix, 0, sizeof(uint64_t) * (size_t)n_sets * n_db, st);
          cudaMemsetAsync(P.ticket, 0, sizeof(uint32_t), st);
          cudaEventRecord(e0, st);
          k_allpairs<<<grid, kApBlock, smem, st>>>(P);
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
      ap_chunk_record(total_q, total_db, n_db, n_sets, (int)chunk);
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
    cudaMemsetAsync(d_matrix, 0, sizeof(uint64_t) * (size_t)n_sets * n_db, cap);
    cudaMemsetAsync(P.ticket, 0, sizeof(uint32_t), cap);
    k_allpairs<<<grid, kApBlock, smem, cap>>>(P);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture(count_matrix)");
    g->graph = graph;
    BITS_CUDA_TRY(cudaGraphInstantiate(&g->exec, graph, 0));
    g->kernels = 1;
    g_graphs.put(key, g);
  }
  BITS_CUDA_TRY(cudaGraphLaunch(g->exec, st));
  count_launch((uint32_t)g->kernels);
  return BITS_OK;
}

void release_matrix_graphs(const bits_db* db) {
  g_graphs.erase_if([db](const std::vector<uint64_t>& key) {
    for (size_t k = 1; k < key.size(); ++k)
      if (key[k] == reinterpret_cast<uintptr_t>(db)) return true;
    return false;
  });
}

}  // namespace bits
