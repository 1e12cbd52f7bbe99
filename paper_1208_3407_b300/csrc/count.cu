// bits_count kernels: Algorithm 2's counting loop over Algorithm 1 (ICount).
//
// One thread per query (Sec. "Parallel BITS" assigns one ICount per thread): a coalesced
// 8-byte load of (start, end), the two top-level searches in shared memory,
// the octet descent through the 16-ary levels (below: one load instruction
// reads both of a query's nodes), a coalesced 4-byte store of
// the count, and a block reduction of the 64-bit total with one atomic per
// CTA.
//
// The tree the searches descend is written by levels.cu.
#include "count.cuh"
#include "search.cuh"

namespace bits {
namespace {

// x[i] for a lane-dependent i < 8 (a select chain: registers cannot be
// indexed at run time).
__device__ __forceinline__ uint32_t select8(const uint32_t (&x)[8], uint32_t i) {
  uint32_t r = x[0];
  #pragma unroll
  for (int o = 1; o < 8; ++o) r = i == (uint32_t)o ? x[o] : r;
  return r;
}

// Octet descent: the same searches as quad_descend (both enter at the top
// level J), with the two nodes of one query read by ONE load instruction.
// Eight lanes own eight queries; lanes 0-3 of the octet walk the starts'
// node of query o and lanes 4-7 the ends' node of the same query, so the
// instruction covers line is and line ie of the interleaved copy, which are
// one 128-byte line when the two searches share their node index (nearly
// always on the upper levels; at level 0 when the query's count is small).
// This part serves a random line read by one instruction at the rate of a
// single 64-byte node, and the same line read by two loads at half of it
// (the random-read probe, access kinds 2 and 3), so each shared index saves
// one memory request.  Used where the searches are bound by memory requests
// (databases far larger than L2); the quad descent stays where instruction
// issue binds.
__device__ __forceinline__ void octet_descend(const LevelIndex& L, uint32_t& is_out,
                                              uint32_t key_s, uint32_t& ie_out, uint32_t key_e,
                                              bool stream_level0 = true) {
  const unsigned lane = lane_id(), sub = lane & 3u, half = (lane >> 2) & 1u;
  const unsigned obase = lane & ~7u;
  const uint64_t pol_last = policy_evict_last();
  const uint64_t pol_first = stream_level0 ? policy_evict_first() : pol_last;
  // Gather: a starts lane needs (is, key_s) of each query of its octet, an
  // ends lane (ie, key_e).  After swapping the ends' pair with lane ^ 4, one
  // shuffle per query and value serves both halves: for queries 0-3 the
  // starts lanes read lane o and the ends lanes lane o + 4 (which then holds
  // query o's ends pair); for queries 4-7 the other way round.
  const uint32_t x_ie = __shfl_xor_sync(0xFFFFFFFFu, ie_out, 4);
  const uint32_t x_ke = __shfl_xor_sync(0xFFFFFFFFu, key_e, 4);
  const uint32_t lo_r = half ? x_ie : is_out, lo_k = half ? x_ke : key_s;
  const uint32_t hi_r = half ? is_out : x_ie, hi_k = half ? key_s : x_ke;
  uint32_t ix[8], kx[8];
  #pragma unroll
  for (int o = 0; o < 8; ++o) {
    const unsigned src = obase | (unsigned)(half ? (o ^ 4) : o);
    ix[o] = __shfl_sync(0xFFFFFFFFu, o < 4 ? lo_r : hi_r, src);
    kx[o] = __shfl_sync(0xFFFFFFFFu, o < 4 ? lo_k : hi_k, src);
  }
  #pragma unroll
  for (int j = kMaxLevels - 1; j >= 1; --j) {
    if (j > L.J) continue;
    const uint32_t lenj = L.len[j], lenm = L.len[j - 1];
    // Node i of level j - 1: starts at il + 32 i, ends at il + 32 i + 16.
    const uint32_t* LX = L.il[j - 1] + 16u * half + 4u * sub;
    const uint64_t pol = j == 1 ? pol_first : pol_last;
    uint4 v[8];
    #pragma unroll
    for (int o = 0; o < 8; ++o)
      v[o] = ix[o] < lenj ? ldg4_hint(LX + 32u * ix[o], pol)
                          : make_uint4(kU32Max, kU32Max, kU32Max, kU32Max);
    #pragma unroll
    for (int o = 0; o < 8; ++o) {
      uint32_t c = cnt4(v[o], kx[o]);
      c += __shfl_xor_sync(0xFFFFFFFFu, c, 1);
      c += __shfl_xor_sync(0xFFFFFFFFu, c, 2);
      ix[o] = ix[o] < lenj ? 16u * ix[o] + c : lenm;
    }
  }
  // Scatter back: lane o of the octet takes its starts rank from a starts
  // lane and its ends rank from an ends lane, mirroring the gather.
  const uint32_t o = lane & 7u;
  const uint32_t a = __shfl_sync(0xFFFFFFFFu, select8(ix, o), obase | o);
  const uint32_t b = __shfl_sync(0xFFFFFFFFu, select8(ix, o ^ 4u), obase | (o ^ 4u));
  is_out = o < 4u ? a : b;
  ie_out = o < 4u ? b : a;
}


// Zeroes the total that k_count_search accumulates into, then lets the
// count kernel, launched right behind it as a programmatic dependent, start
// at once: the count kernel stages its top level and runs its searches while
// this grid drains, and waits for it (griddepcontrol.wait) only before its
// one atomic on the total.
__global__ void k_zero_total(unsigned long long* __restrict__ total) {
  if (threadIdx.x == 0) *total = 0ull;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// BLOCK threads per CTA and 1024 / BLOCK CTAs per SM (64 registers); the
// autotuner picks BLOCK.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK)
k_count_search(const uint2* __restrict__ a, uint32_t n, LevelIndex L, uint32_t nb,
               uint32_t* __restrict__ counts, unsigned long long* __restrict__ total,
               uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) uint32_t s_top[];
  __shared__ unsigned long long s_red[32];
  const uint32_t stride = gridDim.x * blockDim.x;
  load_top(s_top, L);
  __syncthreads();
  unsigned long long acc = 0ull;
  bool bad = false;
  // 64-bit indices: n may come within one grid stride of 2^32.
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const uint64_t i = base + threadIdx.x;
    const bool valid = i < n;
    uint2 q = make_uint2(0u, 0u);
    if (valid) q = __ldcs(a + i);
    const uint32_t key_s = q.y, key_e = q.x + 1u;
    uint32_t rs, re;
    top_rank2(s_top, L.top_size, key_s, key_e, rs, re);
    octet_descend(L, rs, key_s, re, key_e);
    uint32_t c = icount_from_ranks(rs, re, q.x, nb);
    if (q.y < q.x) {
      c = 0u;
      bad = true;
    }
    if (valid) {
      if (counts) __stcs(counts + i, c);
      acc += c;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_dev_error(err, DEV_ERR_INVALID);
  const unsigned long long sum = block_sum_u64(acc, s_red);
  grid_dependency_wait();
  if (threadIdx.x == 0 && sum) atomicAdd(total, sum);
}

template <int BLOCK>
bits_status launch_search(const LevelIndex& L, const bits_db* db, const uint2* a, uint32_t n,
                          uint32_t* d_counts, uint64_t* d_total, cudaStream_t st) {
  const size_t smem = sizeof(uint32_t) * 2 * top_words(L.top_size);
  const int per_sm = kernel_blocks_per_sm(reinterpret_cast<const void*>(k_count_search<BLOCK>),
                                          BLOCK, smem);
  const uint32_t need = (n + BLOCK - 1) / BLOCK;
  const uint32_t grid = std::min<uint32_t>(need, (uint32_t)(per_sm * sm_count()));
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  pdl_config(cfg, attr, dim3(grid), dim3(BLOCK), smem, st);
  BITS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_count_search<BLOCK>, a, n, L, db->n, d_counts,
                                   reinterpret_cast<unsigned long long*>(d_total), db->err));
  BITS_LAUNCH_CHECK("k_count_search");
  return BITS_OK;
}

}  // namespace

bits_status launch_zero_total(uint64_t* d_total, cudaStream_t st) {
  k_zero_total<<<1, 32, 0, st>>>(reinterpret_cast<unsigned long long*>(d_total));
  BITS_LAUNCH_CHECK("k_zero_total");
  return BITS_OK;
}

bits_status launch_count_search(const bits_db* db, const uint32_t* d_a, uint32_t n,
                                uint32_t* d_counts, uint64_t* d_total, cudaStream_t st,
                                const TuneCount* tc) {
  bits_status s = launch_zero_total(d_total, st);
  if (s != BITS_OK || n == 0) return s;
  const TuneCount t = tc ? *tc : count_params(db, BITS_METHOD_SEARCH, n, d_counts != nullptr);
  const LevelIndex L = level_view(db, t.raise);
  const uint2* a = reinterpret_cast<const uint2*>(d_a);
  return t.block == 256 ? launch_search<256>(L, db, a, n, d_counts, d_total, st)
                        : launch_search<512>(L, db, a, n, d_counts, d_total, st);
}

}  // namespace bits
