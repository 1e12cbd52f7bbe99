// Monte-Carlo screen over many query sets and databases (Sec. "Novel genomic relationships": every
// pair of the 159 tracks, 1e4 shuffles each).  For query set i and database
// j, totals[i][j][s] is the count of set i re-placed by shuffle s against
// database j, the observed matrix is bits_count_matrix's, and the optional
// summary gives each pair's tallies and Fig. 3 enrichment score.
//
// One persistent launch covers every pair.  A task is one (database, set)
// pair; its work units are (chunk of kMcChunk intervals, block of kMcBlock
// shuffles), the unit of the single-test kernel.  Tasks are ordered database
// by database, largest database first, so the deepest searches start early
// and a CTA mostly stays on one database: it reloads the shared-memory top
// level only when its unit's database changes.  CTAs take units from an
// atomic ticket and find the unit's task by binary search over the tasks'
// unit prefix sums.  Set i draws Philox at counter (interval, shuffle, i, 0),
// so its placements are the same against every database and set 0's are
// the single test's.
//
// Because of that, one shuffle's totals for every pair are the all-pairs
// matrix of the shuffle's placed sets against the databases.  When it pays
// (the sets' placements searched against every database cost at least
// twice as much as building the placed sets as databases and counting each
// pair from its smaller side) and every query interval is non-empty and
// inside its contig, the screen runs that way instead: per shuffle,
// k_mc_place writes each set's placed intervals, the placed set is sorted
// into a database of its own (built on the first shuffle, rebuilt in the
// same memory afterwards), run_count_matrix_db counts the matrix
// (allpairs.cu), and k_mc_scatter stores it as that shuffle's totals.  The
// placements are the same Philox draws, so the totals are the same.
#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "allpairs.cuh"
#include "philox.cuh"
#include "mc_matrix.cuh"
#include "mc_stats.cuh"
#include "mc_unit.cuh"

namespace bits {
namespace {

struct McDb {
  LevelIndex L;
  uint32_t nb;
  uint32_t* err;
};

struct McTask {
  uint32_t db, set, n, chunks;
  unsigned long long row;  // first total of this pair: (set * n_db + db) * n_shuffles
};

struct McMatArgs {
  const McDb* dbs;
  const McTask* tasks;
  const uint32_t* prefix;  // [n_tasks + 1] unit prefix sums
  uint32_t n_tasks, n_units;
  const uint2* const* sets;
  const uint32_t* coff;
  const uint32_t* clen;
  uint32_t nc, nc_pad;  // contigs; table slots in shared memory (a multiple of 4)
  uint32_t key0, key1;
  uint32_t s_begin, n_shuffles;
  unsigned long long* totals;
  uint32_t* ticket;
};

__global__ void __launch_bounds__(kMcBlock)
k_mc_matrix(McMatArgs P) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ McDb s_db;
  __shared__ McTask s_task;
  __shared__ uint32_t s_unit, s_local;
  __shared__ int s_cur;
  uint32_t* s_coff = smem;
  uint32_t* s_clen = s_coff + P.nc_pad;
  uint32_t* s_off = s_clen + P.nc_pad;
  uint32_t* s_rng = s_off + kMcChunk;
  uint32_t* s_len = s_rng + kMcChunk;
  uint32_t* s_top = s_len + kMcChunk;

  for (uint32_t c = threadIdx.x; c < P.nc; c += blockDim.x) {
    s_coff[c] = P.coff[c];
    s_clen[c] = P.clen[c];
  }
  if (threadIdx.x == 0) s_cur = -1;
  const RmiView R{};
  bool bad = false;
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t u = atomicAdd(P.ticket, 1u);
      s_unit = u;
      if (u < P.n_units) {
        uint32_t lo = 0, hi = P.n_tasks;  // last task with prefix <= u
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (P.prefix[mid] <= u) lo = mid; else hi = mid;
        }
        s_task = P.tasks[lo];
        s_local = u - P.prefix[lo];
      }
    }
    __syncthreads();
    if (s_unit >= P.n_units) break;
    const McTask T = s_task;
    const uint32_t local = s_local;
    if ((int)T.db != s_cur) {
      if (bad) set_dev_error(s_db.err, DEV_ERR_INVALID);  // flag the database it came from
      bad = false;
      __syncthreads();
      const uint32_t* src = reinterpret_cast<const uint32_t*>(P.dbs + T.db);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&s_db);
      for (uint32_t k = threadIdx.x; k < sizeof(McDb) / 4; k += blockDim.x) dst[k] = src[k];
      __syncthreads();
      load_top(s_top, s_db.L);
      if (threadIdx.x == 0) s_cur = (int)T.db;
    }
    const uint32_t chunk = local % T.chunks, sb = local / T.chunks;
    const uint32_t i0 = chunk * kMcChunk;
    const uint32_t cn = min((uint32_t)kMcChunk, T.n - i0);
    mc_stage_chunk(P.sets[T.set], i0, cn, s_coff, s_clen, P.nc, s_off, s_len, s_rng, bad);
    __syncthreads();
    const McLane ln = mc_lane(sb, P.n_shuffles);
    const unsigned long long acc =
        mc_count_chunk<false>(s_top, s_db.L, R, s_db.nb, s_off, s_len, s_rng, i0, cn, ln,
                              P.s_begin + ln.s_local, T.set, P.key0, P.key1);
    if (ln.active && acc) atomicAdd(P.totals + T.row + ln.s_local, acc);
    __syncthreads();  // the unit's shared state is free again
  }
  if (bad && s_cur >= 0) set_dev_error(s_db.err, DEV_ERR_INVALID);
}

int mcm_blocks_per_sm(size_t smem) {
  return kernel_blocks_per_sm(reinterpret_cast<const void*>(k_mc_matrix), kMcBlock, smem,
                              kMcCtasPerSm);
}

struct McMatGraph {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  void* dev = nullptr;  // databases | tasks | prefix | set pointers | ticket
  ~McMatGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (dev) cudaFree(dev);
  }
};

// At most 16 argument sets keep a captured graph (graph_cache.cuh).
GraphCache<std::vector<uint64_t>, McMatGraph> g_graphs(16);

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// ---- the screen by databases on both sides --------------------------------

constexpr int kPlaceBlock = 256;

// Sets *flag unless every interval is non-empty and inside its contig.
__global__ void __launch_bounds__(kPlaceBlock)
k_mc_screen_check(const uint2* __restrict__ A, uint32_t n, const uint32_t* __restrict__ coff,
                  const uint32_t* __restrict__ clen, uint32_t nc, uint32_t* __restrict__ flag) {
  bool bad = false;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint2 q = A[k];
    const int c = contig_of(coff, nc, q.x);
    bad |= !(c >= 0 && q.y > q.x &&
             (unsigned long long)q.y <= (unsigned long long)coff[c] + clen[c]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1u);
}

// Interval k of set `set` placed by shuffle s: the draw and the offset of
// mc_count_chunk (mc_unit.cuh), written out as an interval.
__global__ void __launch_bounds__(kPlaceBlock)
k_mc_place(const uint2* __restrict__ A, uint32_t n, uint32_t set, uint32_t s, uint32_t key0,
           uint32_t key1, const uint32_t* __restrict__ coff, const uint32_t* __restrict__ clen,
           uint32_t nc, uint2* __restrict__ out) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint2 q = A[k];
    const int c = contig_of(coff, nc, q.x);  // valid: checked by k_mc_screen_check
    const uint32_t len = q.y - q.x;
    const uint32_t rng = clen[c] - len + 1u;
    const uint4 x = philox4x32_10(make_uint4(k, s, set, 0u), key0, key1);
    const uint32_t start = coff[c] + philox_offset(x, rng);
    out[k] = make_uint2(start, start + len);
  }
}

// totals[p][s_local] = m[p] for every pair p.
__global__ void k_mc_scatter(const unsigned long long* __restrict__ m, uint32_t n_pairs,
                             uint32_t n_shuffles, uint32_t s_local,
                             unsigned long long* __restrict__ totals) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n_pairs) totals[(size_t)p * n_shuffles + s_local] = m[p];
}

// Whether the screen by databases pays: the persistent kernel searches every
// placement in every database; the other way builds each placed set (about
// four searches' worth of work per interval, measured) and counts each pair
// from its smaller side.  Small screens stay with the persistent kernel.
bool screen_by_databases_pays(const bits_db* const* dbs, uint32_t n_db, const uint64_t* n_as,
                              uint32_t n_sets) {
  uint64_t sum_a = 0, pairs_min = 0;
  for (uint32_t i = 0; i < n_sets; ++i) {
    sum_a += n_as[i];
    for (uint32_t j = 0; j < n_db; ++j) pairs_min += std::min<uint64_t>(n_as[i], dbs[j]->n);
  }
  if (sum_a < (1u << 20)) return false;
  return 2 * (pairs_min + 4 * sum_a) < sum_a * n_db;
}

// The observed matrix and every shuffle's totals by databases on both sides,
// unless an interval is empty or outside its contig (*taken = false: nothing
// was written).  The sets are built as databases from their own intervals
// (the observed matrix), then rebuilt in the same memory from each shuffle's
// placements.
bits_status run_screen_by_databases(const bits_db* const* dbs, uint32_t n_db,
                                    const uint32_t* const* d_as, const uint64_t* n_as,
                                    uint32_t n_sets, const uint32_t* coff, const uint32_t* clen,
                                    uint32_t nc, uint64_t seed, uint32_t s_begin, uint32_t s_end,
                                    uint64_t* d_observed, uint64_t* d_totals, cudaStream_t st,
                                    bool* taken) {
  *taken = false;
  uint64_t max_n = 1;
  for (uint32_t i = 0; i < n_sets; ++i) max_n = std::max<uint64_t>(max_n, n_as[i]);
  const size_t off_flag = align256(sizeof(uint2) * max_n);
  const size_t off_m = off_flag + 256;
  const size_t bytes = off_m + sizeof(uint64_t) * (size_t)n_sets * n_db;
  void* scratch = nullptr;
  {
    const bits_status as = pool_alloc(&scratch, bytes, st);
    if (as != BITS_OK) return as;
  }
  uint2* placed = static_cast<uint2*>(scratch);
  uint32_t* d_flag = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch) + off_flag);
  uint64_t* d_m = reinterpret_cast<uint64_t*>(static_cast<char*>(scratch) + off_m);
  std::vector<bits_db*> sets(n_sets, nullptr);
  auto finish = [&](bits_status s) {
    for (bits_db* d : sets) bits_free(d);
    pool_free(scratch, st);
    return s;
  };
  auto grid_for = [](uint64_t n) {
    return (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>((n + kPlaceBlock - 1) / kPlaceBlock, (uint64_t)sm_count() * 8));
  };
  // Every interval non-empty and inside its contig (one read-back).
  BITS_CUDA_TRY(cudaMemsetAsync(d_flag, 0, sizeof(uint32_t), st));
  for (uint32_t i = 0; i < n_sets; ++i)
    if (n_as[i]) {
      k_mc_screen_check<<<grid_for(n_as[i]), kPlaceBlock, 0, st>>>(
          reinterpret_cast<const uint2*>(d_as[i]), (uint32_t)n_as[i], coff, clen, nc, d_flag);
      count_launch();
    }
  uint32_t h_flag = 0;
  BITS_CUDA_TRY(cudaMemcpyAsync(&h_flag, d_flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  BITS_CUDA_TRY(cudaStreamSynchronize(st));
  if (h_flag) return finish(BITS_OK);  // left to the persistent kernel, which flags it
  *taken = true;
  const uint32_t n_pairs = n_sets * n_db;
  for (uint32_t i = 0; i < n_sets; ++i) {
    const bits_status b = bits_build_db(n_as[i] ? d_as[i] : nullptr, n_as[i], nullptr,
                                        static_cast<void*>(st), &sets[i]);
    if (b != BITS_OK) return finish(b);
  }
  {
    const bits_status c = run_count_matrix_db(sets.data(), n_sets, dbs, n_db, d_m, st);
    if (c != BITS_OK) return finish(c);
    BITS_CUDA_TRY(cudaMemcpyAsync(d_observed, d_m, sizeof(uint64_t) * n_pairs,
                                  cudaMemcpyDeviceToDevice, st));
  }
  const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
  const uint32_t n_shuffles = s_end - s_begin;
  for (uint32_t s = s_begin; s < s_end; ++s) {
    for (uint32_t i = 0; i < n_sets; ++i) {
      if (!n_as[i]) continue;
      k_mc_place<<<grid_for(n_as[i]), kPlaceBlock, 0, st>>>(
          reinterpret_cast<const uint2*>(d_as[i]), (uint32_t)n_as[i], i, s, key0, key1, coff,
          clen, nc, placed);
      count_launch();
      const bits_status b = db_rebuild(sets[i], reinterpret_cast<const uint32_t*>(placed), st);
      if (b != BITS_OK) return finish(b);
    }
    bits_status c = run_count_matrix_db(sets.data(), n_sets, dbs, n_db, d_m, st);
    if (c != BITS_OK) return finish(c);
    k_mc_scatter<<<(n_pairs + 255) / 256, 256, 0, st>>>(
        reinterpret_cast<const unsigned long long*>(d_m), n_pairs, n_shuffles, s - s_begin,
        reinterpret_cast<unsigned long long*>(d_totals));
    count_launch();
  }
  return finish(BITS_OK);
}

}  // namespace

bits_status run_mc_matrix(const bits_db* const* dbs, uint32_t n_db, const uint32_t* const* d_as,
                          const uint64_t* n_as, uint32_t n_sets, const uint32_t* d_contig_off,
                          const uint32_t* d_contig_len, uint32_t n_contigs, uint64_t seed,
                          uint32_t shuffle_begin, uint32_t shuffle_end, uint64_t* d_observed,
                          uint64_t* d_totals, bits_mc_stat* d_stats, cudaStream_t st) {
  const uint32_t n_shuffles = shuffle_end - shuffle_begin;
  if (n_db == 0 || n_sets == 0) return BITS_OK;
  bits_status s;
  if (n_shuffles && n_contigs && screen_by_databases_pays(dbs, n_db, n_as, n_sets)) {
    bool taken = false;
    s = run_screen_by_databases(dbs, n_db, d_as, n_as, n_sets, d_contig_off, d_contig_len,
                                n_contigs, seed, shuffle_begin, shuffle_end, d_observed, d_totals,
                                st, &taken);
    if (s != BITS_OK) return s;
    if (taken) {
      if (d_stats)
        return launch_mc_summary(d_totals, n_shuffles, n_sets * n_db, d_observed, d_stats, st);
      return BITS_OK;
    }
  }
  // Observed matrix: Algorithm 2 for every pair (the all-pairs kernel).
  s = run_count_matrix(dbs, n_db, d_as, n_as, n_sets, d_observed, st);
  if (s != BITS_OK) return s;
  std::vector<uint64_t> key = {reinterpret_cast<uintptr_t>(d_totals), seed, shuffle_begin,
                               shuffle_end, reinterpret_cast<uintptr_t>(d_contig_off),
                               reinterpret_cast<uintptr_t>(d_contig_len), n_contigs};
  for (uint32_t j = 0; j < n_db; ++j) key.push_back(reinterpret_cast<uintptr_t>(dbs[j]));
  for (uint32_t i = 0; i < n_sets; ++i) {
    key.push_back(reinterpret_cast<uintptr_t>(d_as[i]));
    key.push_back(n_as[i]);
  }
  std::shared_ptr<McMatGraph> g = g_graphs.find(key);
  if (!g && n_shuffles) {
    std::vector<McDb> hd(n_db);
    size_t max_top = 4;
    for (uint32_t j = 0; j < n_db; ++j) {
      hd[j].L = dbs[j]->lvl;
      hd[j].nb = dbs[j]->n;
      hd[j].err = dbs[j]->err;
      max_top = std::max<size_t>(max_top, top_words(dbs[j]->lvl.top_size));
    }
    std::vector<uint32_t> order(n_db);
    for (uint32_t j = 0; j < n_db; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t x, uint32_t y) { return dbs[x]->n > dbs[y]->n; });
    const uint64_t n_sblocks = (n_shuffles + kMcBlock - 1) / kMcBlock;
    std::vector<McTask> tasks;
    std::vector<uint32_t> prefix(1, 0);
    uint64_t total_units = 0;
    for (uint32_t j : order)
      for (uint32_t i = 0; i < n_sets; ++i) {
        if (n_as[i] == 0) continue;
        const uint64_t chunks = (n_as[i] + kMcChunk - 1) / kMcChunk;
        tasks.push_back(McTask{j, i, (uint32_t)n_as[i], (uint32_t)chunks,
                               ((unsigned long long)i * n_db + j) * n_shuffles});
        total_units += chunks * n_sblocks;
        if (total_units >= (1ull << 32)) {
          set_error("bits_mc_matrix: more than 2^32 work units; split the shuffle range");
          return BITS_EOVERFLOW;
        }
        prefix.push_back((uint32_t)total_units);
      }
    g = std::make_shared<McMatGraph>();
    const size_t nt = std::max<size_t>(tasks.size(), 1);
    const size_t off_tasks = align256(sizeof(McDb) * n_db);
    const size_t off_prefix = off_tasks + align256(sizeof(McTask) * nt);
    const size_t off_sets = off_prefix + align256(sizeof(uint32_t) * (nt + 1));
    const size_t off_ticket = off_sets + align256(sizeof(void*) * n_sets);
    BITS_CUDA_TRY(cudaMalloc(&g->dev, off_ticket + 256));
    char* base = static_cast<char*>(g->dev);
    std::vector<const void*> sets(d_as, d_as + n_sets);
    BITS_CUDA_TRY(cudaMemcpy(base, hd.data(), sizeof(McDb) * n_db, cudaMemcpyHostToDevice));
    if (!tasks.empty())
      BITS_CUDA_TRY(cudaMemcpy(base + off_tasks, tasks.data(), sizeof(McTask) * tasks.size(),
                               cudaMemcpyHostToDevice));
    BITS_CUDA_TRY(cudaMemcpy(base + off_prefix, prefix.data(), sizeof(uint32_t) * prefix.size(),
                             cudaMemcpyHostToDevice));
    BITS_CUDA_TRY(cudaMemcpy(base + off_sets, sets.data(), sizeof(void*) * n_sets,
                             cudaMemcpyHostToDevice));
    McMatArgs P{};
    P.dbs = reinterpret_cast<const McDb*>(base);
    P.tasks = reinterpret_cast<const McTask*>(base + off_tasks);
    P.prefix = reinterpret_cast<const uint32_t*>(base + off_prefix);
    P.n_tasks = (uint32_t)tasks.size();
    P.n_units = (uint32_t)total_units;
    P.sets = reinterpret_cast<const uint2* const*>(base + off_sets);
    P.coff = d_contig_off;
    P.clen = d_contig_len;
    P.nc = n_contigs;
    P.nc_pad = (n_contigs + 3) & ~3u;
    P.key0 = (uint32_t)seed;
    P.key1 = (uint32_t)(seed >> 32);
    P.s_begin = shuffle_begin;
    P.n_shuffles = n_shuffles;
    P.totals = reinterpret_cast<unsigned long long*>(d_totals);
    P.ticket = reinterpret_cast<uint32_t*>(base + off_ticket);
    const size_t smem = sizeof(uint32_t) * (2 * P.nc_pad + 3 * kMcChunk + 2 * max_top);
    const uint32_t grid = std::min<uint32_t>(std::max<uint32_t>(P.n_units, 1),
                                             (uint32_t)(mcm_blocks_per_sm(smem) * sm_count()));
    cudaStream_t cap = nullptr;
    BITS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_status(e, "cudaStreamBeginCapture");
    }
    cudaMemsetAsync(d_totals, 0, sizeof(uint64_t) * (size_t)n_sets * n_db * n_shuffles, cap);
    cudaMemsetAsync(P.ticket, 0, sizeof(uint32_t), cap);
    k_mc_matrix<<<grid, kMcBlock, smem, cap>>>(P);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture(mc_matrix)");
    g->graph = graph;
    BITS_CUDA_TRY(cudaGraphInstantiate(&g->exec, graph, 0));
    g_graphs.put(key, g);
  }
  if (g) {
    BITS_CUDA_TRY(cudaGraphLaunch(g->exec, st));
    count_launch(1);
  }
  if (d_stats)
    return launch_mc_summary(d_totals, n_shuffles, n_sets * n_db, d_observed, d_stats, st);
  return BITS_OK;
}

void release_mc_matrix_graphs(const bits_db* db) {
  g_graphs.erase_if([db](const std::vector<uint64_t>& key) {
    for (size_t k = 7; k < key.size(); ++k)
      if (key[k] == reinterpret_cast<uintptr_t>(db)) return true;
    return false;
  });
}

}  // namespace bits
