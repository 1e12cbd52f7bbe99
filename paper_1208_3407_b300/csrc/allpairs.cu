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
// L2.  Units are as above with the larger side as the database.  Pairs whose
// sides are within a factor kMergeRatio in size skip the searches: both rank
// sums are read off merges of the sorted arrays (k_merge_splits,
// k_merge_sums below), which read each array once.
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

// ---- rank sums by merge path (bits_count_matrix_db, pairs of similar size) --
//
// For sorted X and Y, sum_{x in X} #(Y < x) (strict) or #(Y <= x) is read off
// the merge of the two arrays in which an element of Y goes before x exactly
// when it is counted: each x adds the number of Y elements merged before it.
// The merge is cut into tiles of kMgTile merged positions; a tile boundary at
// diagonal d splits it into the first i elements of X and d - i of Y (merge
// path: the binary search of merge_split).  A CTA stages one tile's X and Y
// elements in shared memory, each thread finds its own diagonal in the tile
// and merges kMgPer positions sequentially.  Both arrays are read once.
constexpr int kMgBlock = 256;
constexpr uint32_t kMgTile = 4096;                 // merged positions per tile
constexpr uint32_t kMgPer = kMgTile / kMgBlock;   // per thread

struct MergeJob {
  const uint32_t* x;
  const uint32_t* y;
  uint32_t nx, ny;
  uint32_t strict;       // 1: counts #(Y < x); 0: #(Y <= x)
  uint32_t negate;       // the sum is subtracted from the entry
  uint32_t out;          // matrix entry
  uint32_t first_tile;   // its first tile among all jobs' tiles
  uint32_t first_split;  // its first tile boundary (tiles + 1 per job)
};

struct MergeArgs {
  const MergeJob* jobs;
  uint32_t n_jobs, n_tiles, n_splits;
  uint32_t* splits;
  unsigned long long* matrix;
};

// x goes before y in the merge: y is not counted for x.
__device__ __forceinline__ bool x_first(uint32_t x, uint32_t y, bool strict) {
  return strict ? x <= y : x < y;
}

// Elements of X among the first d merged positions.
template <typename P>
__device__ __forceinline__ uint32_t merge_split(P X, uint32_t nx, P Y, uint32_t ny, uint64_t d,
                                                bool strict) {
  uint32_t lo = d > ny ? (uint32_t)(d - ny) : 0u;
  uint32_t hi = (uint32_t)(d < nx ? d : nx);
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (x_first(X[mid], Y[d - mid - 1], strict)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Last job whose field `first` is <= v (jobs ordered by it).
__device__ __forceinline__ uint32_t find_job(const MergeJob* jobs, uint32_t n, uint32_t v,
                                             bool by_tile) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    const uint32_t f = by_tile ? jobs[mid].first_tile : jobs[mid].first_split;
    if (f <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void k_merge_splits(MergeArgs P) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < P.n_splits;
       b += gridDim.x * blockDim.x) {
    const MergeJob J = P.jobs[find_job(P.jobs, P.n_jobs, b, false)];
    const uint64_t total = (uint64_t)J.nx + J.ny;
    const uint64_t d = min((uint64_t)(b - J.first_split) * kMgTile, total);
    P.splits[b] = merge_split(J.x, J.nx, J.y, J.ny, d, J.strict != 0);
  }
}

// One tile's place in its merge.
struct MgTile {
  uint32_t job, i0, j0, lx, ly;
};

__device__ __forceinline__ MgTile tile_of(const MergeArgs& P, uint32_t& jb, uint32_t t) {
  while (jb + 1 < P.n_jobs && P.jobs[jb + 1].first_tile <= t) ++jb;
  const MergeJob& J = P.jobs[jb];
  const uint32_t k = t - J.first_tile;
  const uint64_t total = (uint64_t)J.nx + J.ny;
  const uint64_t d0 = (uint64_t)k * kMgTile;
  const uint64_t d1 = min(d0 + kMgTile, total);
  const uint32_t i0 = P.splits[J.first_split + k], i1 = P.splits[J.first_split + k + 1];
  const uint32_t j0 = (uint32_t)(d0 - i0), j1 = (uint32_t)(d1 - i1);
  return MgTile{jb, i0, j0, i1 - i0, j1 - j0};
}

__device__ __forceinline__ void cp_async4(uint32_t* dst, const uint32_t* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

// Starts the copy of a tile's X then Y elements into buf (asynchronous).
__device__ __forceinline__ void stage_tile(const MergeArgs& P, const MgTile& T, uint32_t* buf) {
  const MergeJob& J = P.jobs[T.job];
  for (uint32_t e = threadIdx.x; e < T.lx; e += kMgBlock) cp_async4(buf + e, J.x + T.i0 + e);
  for (uint32_t e = threadIdx.x; e < T.ly; e += kMgBlock)
    cp_async4(buf + T.lx + e, J.y + T.j0 + e);
}

__global__ void __launch_bounds__(kMgBlock)
k_merge_sums(MergeArgs P) {
  __shared__ uint32_t s_buf[2][kMgTile];
  __shared__ unsigned long long s_red[32];
  // Each CTA takes a contiguous run of tiles, so it finds a job once and
  // then walks its tiles in order; the next tile streams into the other
  // buffer (cp.async) while this one is merged.
  const uint32_t per = (P.n_tiles + gridDim.x - 1) / gridDim.x;
  const uint32_t t_begin = min(P.n_tiles, blockIdx.x * per);
  const uint32_t t_end = min(P.n_tiles, t_begin + per);
  if (t_begin >= t_end) return;
  uint32_t jb = find_job(P.jobs, P.n_jobs, t_begin, true);
  MgTile cur = tile_of(P, jb, t_begin);
  stage_tile(P, cur, s_buf[0]);
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (uint32_t t = t_begin; t < t_end; ++t) {
    const uint32_t slot = (t - t_begin) & 1u;
    MgTile next{};
    if (t + 1 < t_end) {
      next = tile_of(P, jb, t + 1);
      stage_tile(P, next, s_buf[slot ^ 1u]);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // this tile's copies are done
    __syncthreads();
    const MergeJob& J = P.jobs[cur.job];
    const bool strict = J.strict != 0;
    const uint32_t lx = cur.lx, ly = cur.ly, j0 = cur.j0;
    const uint32_t* sx = s_buf[slot];
    const uint32_t* sy = sx + lx;
    const uint32_t len = lx + ly;
    const uint32_t e0 = min(threadIdx.x * kMgPer, len), e1 = min(e0 + kMgPer, len);
    uint32_t a = merge_split(sx, lx, sy, ly, e0, strict), b = e0 - a;
    unsigned long long sum = 0ull;
    for (uint32_t e = e0; e < e1; ++e) {
      const bool take_x = a < lx && (b >= ly || x_first(sx[a], sy[b], strict));
      if (take_x) {
        sum += j0 + b;  // the Y elements merged before this x
        ++a;
      } else {
        ++b;
      }
    }
    const unsigned long long s = block_sum_u64(sum, s_red);
    if (threadIdx.x == 0 && s) atomicAdd(P.matrix + J.out, J.negate ? 0ull - s : s);
    __syncthreads();  // every thread is done with s_buf[slot] before it is refilled
    cur = next;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <bool kSorted>
int ap_blocks_per_sm(size_t smem) {
  return kernel_blocks_per_sm(reinterpret_cast<const void*>(k_allpairs<kSorted>), kApBlock, smem);
}

struct MatGraph {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  void* dev = nullptr;    // descriptors | units | source pointers | ticket
  void* merge = nullptr;  // merge jobs | tile boundaries (bits_count_matrix_db)
  uint64_t kernels = 0;
  ~MatGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (dev) cudaFree(dev);
    if (merge) cudaFree(merge);
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
                               cudaStream_t st,
                               const std::function<void(cudaStream_t)>& extra = {},
                               uint32_t extra_kernels = 0) {
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
  if (extra) extra(cap);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cap, &graph);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture(count_matrix)");
  g.graph = graph;
  BITS_CUDA_TRY(cudaGraphInstantiate(&g.exec, graph, 0));
  g.kernels = 1 + extra_kernels;
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
    // Pairs of similar size (the larger side at most kMergeRatio times the
    // smaller) are counted by merging the sorted arrays (k_merge_sums):
    // streaming both costs less than searching every key; the others by
    // searches (k_allpairs<true>).
    constexpr uint64_t kMergeRatio = 8;
    std::vector<Pair> pairs;
    std::vector<MergeJob> jobs;
    uint32_t n_tiles = 0, n_splits = 0;
    uint64_t total_keys = 0;
    for (uint32_t i = 0; i < n_a; ++i)
      for (uint32_t j = 0; j < n_b; ++j) {
        const bool a_keys = a_dbs[i]->n <= b_dbs[j]->n;
        const Pair p{a_keys ? n_a + j : i, a_keys ? i : n_a + j,
                     a_keys ? a_dbs[i]->n : b_dbs[j]->n, i * n_b + j};
        if (!p.n) continue;
        const bits_db* K = all[p.src];
        const bits_db* T = all[p.tree];
        if ((uint64_t)T->n <= kMergeRatio * p.n) {
          // total = sum_{x in K_E} #(T_S < x) - sum_{x in K_S} #(T_E <= x)
          const uint32_t tiles = (uint32_t)(((uint64_t)K->n + T->n + kMgTile - 1) / kMgTile);
          jobs.push_back(MergeJob{K->be, T->bs, K->n, T->n, 1u, 0u, p.out, n_tiles, n_splits});
          n_tiles += tiles;
          n_splits += tiles + 1;
          jobs.push_back(MergeJob{K->bs, T->be, K->n, T->n, 0u, 1u, p.out, n_tiles, n_splits});
          n_tiles += tiles;
          n_splits += tiles + 1;
        } else {
          total_keys += p.n;
          pairs.push_back(p);
        }
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
    MergeArgs M{};
    std::function<void(cudaStream_t)> merges;
    if (!jobs.empty()) {
      const size_t off_splits = align256(sizeof(MergeJob) * jobs.size());
      BITS_CUDA_TRY(cudaMalloc(&g->merge, off_splits + sizeof(uint32_t) * (size_t)n_splits));
      BITS_CUDA_TRY(cudaMemcpy(g->merge, jobs.data(), sizeof(MergeJob) * jobs.size(),
                               cudaMemcpyHostToDevice));
      M.jobs = static_cast<const MergeJob*>(g->merge);
      M.n_jobs = (uint32_t)jobs.size();
      M.n_tiles = n_tiles;
      M.n_splits = n_splits;
      M.splits = reinterpret_cast<uint32_t*>(static_cast<char*>(g->merge) + off_splits);
      M.matrix = reinterpret_cast<unsigned long long*>(d_matrix);
      const uint32_t grid_s = std::max<uint32_t>(
          1, std::min<uint32_t>((n_splits + 255) / 256, (uint32_t)sm_count() * 8));
      const int per_sm =
          kernel_blocks_per_sm(reinterpret_cast<const void*>(k_merge_sums), kMgBlock, 0);
      const uint32_t grid_m =
          std::max<uint32_t>(1, std::min<uint32_t>(n_tiles, (uint32_t)(per_sm * sm_count())));
      merges = [M, grid_s, grid_m](cudaStream_t cs) {
        k_merge_splits<<<grid_s, 256, 0, cs>>>(M);
        k_merge_sums<<<grid_m, kMgBlock, 0, cs>>>(M);
      };
    }
    const bits_status s = build_matrix_graph<true>(*g, hd, keys, max_top, make_units,
                                                   "allpairs_db", total_keys, total_db, n_a, d_matrix,
                                                   (size_t)n_a * n_b, st, merges,
                                                   jobs.empty() ? 0u : 2u);
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
