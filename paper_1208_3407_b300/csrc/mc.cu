// Monte-Carlo significance test (Sec. "Monte Carlo Simulations"): each shuffle re-places every
// query interval uniformly inside its own contig (length kept) and recounts
// it against the fixed database; the observed total is the count of the
// unshuffled queries; k_ge = #{s : total_s >= observed}.
//
// k_mc_search is persistent.  A work unit is (chunk of CHUNK intervals,
// block of BLOCK shuffles; 1024 and 256 by default, tuned per size class);
// a thread owns one shuffle, so the block walks the chunk's intervals out of
// shared memory (a broadcast read) and keeps its shuffle's running total in
// a register: one atomic per thread per unit, no reduction tree.  A block
// of fewer than BLOCK shuffles splits the chunk's intervals between groups
// of threads instead (mc_unit.cuh).  Per placement: one Philox4x32-10 block,
// a multiply-high offset, and the two rank searches of search.cuh
// (shared-memory top level, then quad-cooperative 64-byte chunks, which for
// a 1M-interval database all sit in L2).  The interval's contig is found
// when the chunk is staged.
//
// A call runs as a CUDA graph (zero totals, observed count, persistent MC
// launch, tally) captured once per argument set and replayed afterwards.
// The first call of a size class that nothing pins first times the work-unit
// shapes and shared-memory tops of tune.cuh on a reduced shuffle range
// (direct launches, the caller's buffers) and records the fastest.
#include <vector>

#include "count.cuh"
#include "mc.cuh"
#include "mc_unit.cuh"
#include "rmi.cuh"

struct bits_mc_graph {
  std::mutex run_mu;  // one replay at a time: d_scalars is read back after each
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  unsigned long long* d_scalars = nullptr;  // [0] observed, [1] k_ge
  uint64_t kernels_per_replay = 0;
  ~bits_mc_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (d_scalars) cudaFree(d_scalars);
  }
};

namespace bits {
namespace {

struct McArgs {
  const uint2* a;
  uint32_t n;
  const uint32_t* coff;
  const uint32_t* clen;
  uint32_t nc;
  uint32_t key0, key1;
  uint32_t s_begin, n_shuffles;
  unsigned long long* totals;
  uint32_t* err;
  uint32_t nb;
};

template <bool kRmi, int BLOCK, int CHUNK>
__global__ void __launch_bounds__(BLOCK)
k_mc_search(McArgs P, LevelIndex L, RmiView R) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* s_top = smem;
  uint32_t* s_off = s_top + (kRmi ? 0u : 2u * top_words(L.top_size));
  uint32_t* s_rng = s_off + CHUNK;
  uint32_t* s_len = s_rng + CHUNK;
  uint32_t* s_coff = s_len + CHUNK;
  uint32_t* s_clen = s_coff + P.nc;

  if (!kRmi) load_top(s_top, L);
  for (uint32_t c = threadIdx.x; c < P.nc; c += blockDim.x) {
    s_coff[c] = P.coff[c];
    s_clen[c] = P.clen[c];
  }
  const uint32_t n_chunks = (P.n + CHUNK - 1) / CHUNK;
  const uint32_t n_sblocks = (P.n_shuffles + BLOCK - 1) / BLOCK;
  const uint32_t units = n_chunks * n_sblocks;
  bool bad = false;
  for (uint32_t u = blockIdx.x; u < units; u += gridDim.x) {
    const uint32_t chunk = u % n_chunks, sb = u / n_chunks;
    const uint32_t i0 = chunk * CHUNK;
    const uint32_t cn = min((uint32_t)CHUNK, P.n - i0);
    __syncthreads();  // previous unit is done with the staged chunk
    mc_stage_chunk<BLOCK, CHUNK>(P.a, i0, cn, s_coff, s_clen, P.nc, s_off, s_len, s_rng, bad);
    __syncthreads();
    const McLane ln = mc_lane<BLOCK>(sb, P.n_shuffles);
    const unsigned long long acc = mc_count_chunk<kRmi>(s_top, L, R, P.nb, s_off, s_len, s_rng, i0,
                                                        cn, ln, P.s_begin + ln.s_local, 0u, P.key0,
                                                        P.key1);
    if (ln.active && acc) atomicAdd(P.totals + ln.s_local, acc);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_dev_error(P.err, DEV_ERR_INVALID);
}

__global__ void k_mc_tally(const unsigned long long* __restrict__ totals, uint32_t n,
                           unsigned long long* scalars) {
  __shared__ unsigned long long s_red[32];
  const unsigned long long obs = scalars[0];
  unsigned long long k = 0;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) k += totals[i] >= obs;
  k = block_sum_u64(k, s_red);
  if (threadIdx.x == 0) scalars[1] = k;
}

size_t mc_smem_bytes(const LevelIndex& L, uint32_t nc, bool rmi, int chunk) {
  return sizeof(uint32_t) * ((rmi ? 0 : 2 * top_words(L.top_size)) + 3 * (size_t)chunk + 2 * nc);
}

// One persistent Monte-Carlo launch over P's shuffles with shape (BLOCK,
// CHUNK): at most kMcCtasPerSm CTAs of 256 threads' worth per SM, the
// shared-memory carveout fitted to them.
template <bool kRmi, int BLOCK, int CHUNK>
bits_status launch_mc_shape(const McArgs& P, const LevelIndex& L, const RmiView& R,
                            cudaStream_t st) {
  const size_t smem = mc_smem_bytes(L, P.nc, kRmi, CHUNK);
  const uint32_t units = ((P.n + CHUNK - 1) / CHUNK) * ((P.n_shuffles + BLOCK - 1) / BLOCK);
  const int per_sm = kernel_blocks_per_sm(reinterpret_cast<const void*>(k_mc_search<kRmi, BLOCK, CHUNK>),
                                          BLOCK, smem, kMcCtasPerSm * (kMcBlock / BLOCK));
  const uint32_t grid = std::min<uint32_t>(units, (uint32_t)(per_sm * sm_count()));
  k_mc_search<kRmi, BLOCK, CHUNK><<<grid, BLOCK, smem, st>>>(P, L, R);
  BITS_LAUNCH_CHECK("k_mc_search");
  return BITS_OK;
}

template <bool kRmi>
bits_status launch_mc_rmi(const McArgs& P, const LevelIndex& L, const RmiView& R, const TuneMc& t,
                          cudaStream_t st) {
  if (t.shuffles == 128 && t.chunk == 1024) return launch_mc_shape<kRmi, 128, 1024>(P, L, R, st);
  if (t.shuffles == 256 && t.chunk == 512) return launch_mc_shape<kRmi, 256, 512>(P, L, R, st);
  if (t.shuffles == 256 && t.chunk == 2048) return launch_mc_shape<kRmi, 256, 2048>(P, L, R, st);
  if (t.shuffles == 128 && t.chunk == 2048) return launch_mc_shape<kRmi, 128, 2048>(P, L, R, st);
  return launch_mc_shape<kRmi, 256, 1024>(P, L, R, st);
}

bits_status launch_mc(const bits_db* db, int method, const McArgs& P, const TuneMc& t,
                      cudaStream_t st) {
  const RmiView R = db->has_rmi ? rmi_view(db) : RmiView{};
  if (method == BITS_METHOD_RMI) return launch_mc_rmi<true>(P, db->lvl, R, t, st);
  return launch_mc_rmi<false>(P, level_view(db, t.raise), R, t, st);
}

McArgs mc_args(const bits_db* db, const uint32_t* d_a, uint32_t n, const uint32_t* d_contig_off,
               const uint32_t* d_contig_len, uint32_t n_contigs, uint64_t seed,
               uint32_t shuffle_begin, uint32_t n_shuffles, uint64_t* d_totals) {
  McArgs P{};
  P.a = reinterpret_cast<const uint2*>(d_a);
  P.n = n;
  P.coff = d_contig_off;
  P.clen = d_contig_len;
  P.nc = n_contigs;
  P.key0 = (uint32_t)seed;
  P.key1 = (uint32_t)(seed >> 32);
  P.s_begin = shuffle_begin;
  P.n_shuffles = n_shuffles;
  P.totals = reinterpret_cast<unsigned long long*>(d_totals);
  P.err = db->err;
  P.nb = db->n;
  return P;
}

// Time the shapes and tops of tune.cuh on up to 1024 of the call's shuffles
// (direct launches into the caller's totals, which the test itself zeroes
// and rewrites afterwards) and record the fastest for the size class.
bits_status tune_mc(bits_db* db, int method, const McArgs& P0, cudaStream_t st) {
  McArgs P = P0;
  P.n_shuffles = std::min<uint32_t>(P0.n_shuffles, 1024u);
  std::vector<TuneMc> cands;
  const int raises = method == BITS_METHOD_RMI ? 0 : std::min(1, db->plan.Tmax - db->plan.J);
  for (const auto& sh : kMcShapes)
    for (int r = 0; r <= raises; ++r) cands.push_back(TuneMc{sh[0], sh[1], r});
  cudaEvent_t e0, e1;
  BITS_CUDA_TRY(cudaEventCreate(&e0));
  BITS_CUDA_TRY(cudaEventCreate(&e1));
  std::vector<float> best(cands.size(), 1e30f);
  bits_status s = BITS_OK;
  for (int round = 0; round < 3 && s == BITS_OK; ++round)
    for (size_t c = 0; c < cands.size() && s == BITS_OK; ++c) {
      if (cudaEventRecord(e0, st) != cudaSuccess) s = cuda_status(cudaGetLastError(), "tune_mc");
      if (s == BITS_OK) s = launch_mc(db, method, P, cands[c], st);
      float ms = 0.f;
      if (s == BITS_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                           cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        s = cuda_status(cudaGetLastError(), "tune_mc");
      if (round > 0) best[c] = std::min(best[c], ms);  // round 0 warms every shape up
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != BITS_OK) return s;
  size_t b = 0;
  for (size_t c = 1; c < cands.size(); ++c)
    if (best[c] < best[b]) b = c;
  mc_record(db, method, P0.n, cands[b]);
  return BITS_OK;
}

// Enqueue the whole test on `st` (used once, under stream capture).
bits_status enqueue_mc(bits_db* db, int method, const TuneMc& t, const uint32_t* d_a,
                       uint32_t n, const uint32_t* d_contig_off, const uint32_t* d_contig_len,
                       uint32_t n_contigs, uint64_t seed, uint32_t shuffle_begin,
                       uint32_t n_shuffles, uint64_t* d_totals, unsigned long long* d_scalars,
                       cudaStream_t st) {
  if (n_shuffles)
    BITS_CUDA_TRY(cudaMemsetAsync(d_totals, 0, sizeof(uint64_t) * n_shuffles, st));
  // Observed total of the unshuffled queries (Algorithm 2 on A itself).
  bits_status s = method == BITS_METHOD_RMI
                      ? launch_count_rmi(db, d_a, n, nullptr, reinterpret_cast<uint64_t*>(d_scalars), st)
                      : launch_count_search(db, d_a, n, nullptr,
                                            reinterpret_cast<uint64_t*>(d_scalars), st);
  if (s != BITS_OK) return s;
  if (n && n_shuffles) {
    const McArgs P = mc_args(db, d_a, n, d_contig_off, d_contig_len, n_contigs, seed,
                             shuffle_begin, n_shuffles, d_totals);
    s = launch_mc(db, method, P, t, st);
    if (s != BITS_OK) return s;
  }
  k_mc_tally<<<1, 1024, 0, st>>>(reinterpret_cast<const unsigned long long*>(d_totals), n_shuffles,
                                 d_scalars);
  BITS_LAUNCH_CHECK("k_mc_tally");
  return BITS_OK;
}

}  // namespace

bits_status run_mc(bits_db* db, int method, const uint32_t* d_a, uint32_t n,
                   const uint32_t* d_contig_off, const uint32_t* d_contig_len, uint32_t n_contigs,
                   uint64_t seed, uint32_t shuffle_begin, uint32_t shuffle_end, uint64_t* d_totals,
                   uint64_t* h_observed, uint64_t* h_k_ge, double* h_pvalue, cudaStream_t st) {
  if (n_contigs > kMaxContigs) {
    set_error("bits_mc: at most 4096 contigs");
    return BITS_EOVERFLOW;
  }
  if (reinterpret_cast<uintptr_t>(d_a) % 8 || reinterpret_cast<uintptr_t>(d_totals) % 8) {
    set_error("bits_mc: misaligned pointer (queries 8 B, totals 8 B)");
    return BITS_EINVAL;
  }
  const uint32_t n_shuffles = shuffle_end - shuffle_begin;
  // Work-unit shape and shared-memory top: pinned, tuned, or timed now.
  bool tuned = false;
  TuneMc t = mc_params(db, method, n, &tuned);
  if (!tuned && !mc_pinned() && n && n_shuffles && !stream_capturing(st)) {
    bits_status s = tune_mc(db, method,
                            mc_args(db, d_a, n, d_contig_off, d_contig_len, n_contigs, seed,
                                    shuffle_begin, n_shuffles, d_totals),
                            st);
    if (s != BITS_OK) return s;
    t = mc_params(db, method, n, nullptr);
  }
  const bits_db::McKey key(method, (const void*)d_a, (uint64_t)n, (const void*)d_contig_off,
                           (const void*)d_contig_len, n_contigs, seed, shuffle_begin, shuffle_end,
                           (void*)d_totals, (t.shuffles << 20) | (t.chunk << 4) | t.raise);
  std::shared_ptr<bits_mc_graph> g = db->mc_graphs.find(key);
  if (!g) {
    g = std::make_shared<bits_mc_graph>();
    BITS_CUDA_TRY(cudaMalloc(&g->d_scalars, 2 * sizeof(unsigned long long)));
    cudaStream_t cap = nullptr;
    BITS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    const uint64_t before = bits_kernel_launches();
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_status(e, "cudaStreamBeginCapture");
    }
    bits_status s = enqueue_mc(db, method, t, d_a, n, d_contig_off, d_contig_len, n_contigs,
                               seed, shuffle_begin, n_shuffles, d_totals, g->d_scalars, cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (s != BITS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
    g->graph = graph;
    BITS_CUDA_TRY(cudaGraphInstantiate(&g->exec, graph, 0));
    g->kernels_per_replay = bits_kernel_launches() - before;
    uncount_launch(g->kernels_per_replay);
    db->mc_graphs.put(key, g);
  }
  // Concurrent calls with the same arguments share the graph and its result
  // words: replay, read back and check one call at a time.
  std::lock_guard<std::mutex> run_lk(g->run_mu);
  BITS_CUDA_TRY(cudaGraphLaunch(g->exec, st));
  count_launch((uint32_t)g->kernels_per_replay);
  unsigned long long h[2] = {0, 0};
  BITS_CUDA_TRY(cudaMemcpyAsync(h, g->d_scalars, sizeof(h), cudaMemcpyDeviceToHost, st));
  bits_status s = read_device_error(db, st, true);
  if (s != BITS_OK) return s;
  if (h_observed) *h_observed = h[0];
  if (h_k_ge) *h_k_ge = h[1];
  if (h_pvalue) *h_pvalue = (double)(h[1] + 1) / (double)((uint64_t)n_shuffles + 1);
  return BITS_OK;
}

void release_mc_graphs(bits_db* db) {
  db->mc_graphs.erase_if([](const bits_db::McKey&) { return true; });
}

}  // namespace bits
