// Enumeration problem (Sec. "Interval Set Intersection problem": report every
// intersecting pair) with the count as the stopping rule of the scan (Sec. "BITS
// Algorithm": |I(B, a)| terminates the enumeration that a single binary search could
// not).
//
// Offsets: per-query counts (the count kernel) and an exclusive scan into
// uint64 offsets, offsets[n] = number of pairs.  The scan is three plain
// launches -- tile sums, one CTA over the tile sums, tile scans -- so no CTA
// waits on another.
//
// Pairs: the database keeps, when built with BITS_FLAG_ENUMERATE, its
// intervals sorted by start (equal starts in index order) as (end, index)
// pairs.  Every interval meeting a starts before a.end, so it lies left of
// first = #(B_S < a.end) in that order.  One warp serves 32 queries: each
// lane finds its query's ranks with the usual two searches (and checks them
// against the offsets it was given); then the warp walks each query's
// entries right to left, 32 coalesced (end, index) pairs per step, keeps
// those with end > a.start and stops once it has the query's count.  Pairs
// of a query come out in that scan order.
#include "count.cuh"
#include "db.cuh"
#include "enumerate.cuh"
#include "search.cuh"

namespace bits {
namespace {

constexpr int kScanBlock = 256;
constexpr int kScanRows = 16;
constexpr uint32_t kScanTile = kScanBlock * kScanRows;  // counts per tile
constexpr int kEnumBlock = 256;

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v) {
  const unsigned lane = lane_id();
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if ((int)lane >= o) v += y;
  }
  return v;
}

// Phase 1: the sum of each tile of kScanTile counts (rows read coalesced).
__global__ void __launch_bounds__(kScanBlock)
k_scan_reduce(const uint32_t* __restrict__ c, uint32_t n, unsigned long long* __restrict__ part) {
  __shared__ unsigned long long s_red[32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  unsigned long long acc = 0ull;
  #pragma unroll 4
  for (int r = 0; r < kScanRows; ++r) {
    const uint64_t i = base + (uint64_t)r * kScanBlock + threadIdx.x;
    if (i < n) acc += __ldcs(c + i);
  }
  acc = block_sum_u64(acc, s_red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// Phase 2: exclusive scan of the tile sums in place (one CTA of 1024
// threads, 1024 sums per round with a running carry); the grand total goes
// to *total.
__global__ void __launch_bounds__(1024)
k_scan_partials(unsigned long long* __restrict__ part, uint32_t nt,
                unsigned long long* __restrict__ total) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned long long s_carry;
  const unsigned w = threadIdx.x >> 5, lane = lane_id();
  if (threadIdx.x == 0) s_carry = 0ull;
  __syncthreads();
  for (uint32_t base = 0; base < nt; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const unsigned long long v = i < nt ? part[i] : 0ull;
    unsigned long long incl = warp_incl_scan(v);
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) s_w[lane] = warp_incl_scan(s_w[lane]);
    __syncthreads();
    incl += w ? s_w[w - 1] : 0ull;
    const unsigned long long carry = s_carry;
    if (i < nt) part[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + s_w[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = s_carry;
}

// Phase 3: each tile's exclusive scan plus its base from phase 2.
__global__ void __launch_bounds__(kScanBlock)
k_scan_down(const uint32_t* __restrict__ c, uint32_t n, const unsigned long long* __restrict__ part,
            unsigned long long* __restrict__ off) {
  __shared__ unsigned long long s_w[kScanBlock / 32];
  __shared__ unsigned long long s_carry;
  const unsigned w = threadIdx.x >> 5, lane = lane_id();
  if (threadIdx.x == 0) s_carry = part[blockIdx.x];
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  for (int r = 0; r < kScanRows; ++r) {
    const uint64_t i = base + (uint64_t)r * kScanBlock + threadIdx.x;
    const unsigned long long v = i < n ? __ldcs(c + i) : 0ull;
    const unsigned long long incl = warp_incl_scan(v);
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    unsigned long long before = 0ull, row = 0ull;
    #pragma unroll
    for (int k = 0; k < kScanBlock / 32; ++k) {
      before += (k < (int)w) ? s_w[k] : 0ull;
      row += s_w[k];
    }
    const unsigned long long carry = s_carry;
    if (i < n) off[i] = carry + before + incl - v;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + row;
    __syncthreads();
  }
}

// (end, index) of the database in start order, from the sorted indices.
__global__ void k_enum_gather(const uint2* __restrict__ b, const uint32_t* __restrict__ idx,
                              uint32_t n, uint2* __restrict__ out) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t j = idx[k];
    out[k] = make_uint2(b[j].y, j);
  }
}

__global__ void __launch_bounds__(kEnumBlock)
k_enumerate(const uint2* __restrict__ a, uint32_t n, LevelIndex L, uint32_t nb,
            const uint2* __restrict__ E, const unsigned long long* __restrict__ off,
            uint2* __restrict__ pairs, uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) uint32_t s_top[];
  load_top(s_top, L);
  __syncthreads();
  const unsigned lane = lane_id();
  const uint64_t warps = (uint64_t)gridDim.x * (kEnumBlock / 32);
  bool bad = false;
  for (uint64_t g = (uint64_t)blockIdx.x * (kEnumBlock / 32) + (threadIdx.x >> 5); g * 32 < n;
       g += warps) {
    const uint64_t i = g * 32 + lane;
    const bool valid = i < n;
    const uint2 q = valid ? a[i] : make_uint2(0u, 0u);
    const uint32_t key_s = q.y, key_e = q.x + 1u;
    uint32_t rs, re;
    top_rank2(s_top, L.top_size, key_s, key_e, rs, re);
    quad_descend(L, rs, key_s, re, key_e);
    uint32_t c = icount_from_ranks(rs, re, q.x, nb);
    if (q.y < q.x) c = 0u;
    const unsigned long long o0 = valid ? off[i] : 0ull, o1 = valid ? off[i + 1] : 0ull;
    const bool match = o1 - o0 == (unsigned long long)c;
    if (valid && (q.y < q.x || !match)) bad = true;
    const uint32_t cq = (valid && match) ? c : 0u;
    unsigned todo = __ballot_sync(0xFFFFFFFFu, cq > 0u);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1u;
      const uint32_t cnt = __shfl_sync(0xFFFFFFFFu, cq, src);
      const uint32_t as = __shfl_sync(0xFFFFFFFFu, q.x, src);
      const unsigned long long ob = __shfl_sync(0xFFFFFFFFu, o0, src);
      const uint32_t qi = (uint32_t)(g * 32 + (uint32_t)src);
      uint32_t top = __shfl_sync(0xFFFFFFFFu, rs, src);  // entries [0, top) remain
      uint32_t found = 0u;
      while (found < cnt && top > 0u) {  // at most ceil(first / 32) steps
        const bool in = lane < top;
        const uint2 e = in ? __ldg(E + (top - 1u - lane)) : make_uint2(0u, 0u);
        const bool hit = in && e.x > as;
        const unsigned hm = __ballot_sync(0xFFFFFFFFu, hit);
        const uint32_t r = found + (uint32_t)__popc(hm & lanemask_lt());
        if (hit && r < cnt) pairs[ob + r] = make_uint2(qi, e.y);
        found += (uint32_t)__popc(hm);
        top = top > 32u ? top - 32u : 0u;
      }
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_dev_error(err, DEV_ERR_INVALID);
}

int enum_blocks_per_sm(size_t smem) {
  return kernel_blocks_per_sm(reinterpret_cast<const void*>(k_enumerate), kEnumBlock, smem);
}

}  // namespace

bits_status launch_enum_gather(const uint32_t* d_b, const uint32_t* d_idx, uint32_t n, uint2* d_out,
                               cudaStream_t st) {
  if (n == 0) return BITS_OK;
  const uint32_t grid = std::min<uint32_t>((n + 255) / 256, (uint32_t)sm_count() * 8);
  k_enum_gather<<<grid, 256, 0, st>>>(reinterpret_cast<const uint2*>(d_b), d_idx, n, d_out);
  BITS_LAUNCH_CHECK("k_enum_gather");
  return BITS_OK;
}

bits_status run_enumerate_offsets(const bits_db* db, const uint32_t* d_a, uint32_t n,
                                  uint64_t* d_offsets, cudaStream_t st) {
  if (n == 0) {
    BITS_CUDA_TRY(cudaMemsetAsync(d_offsets, 0, sizeof(uint64_t), st));
    return BITS_OK;
  }
  const uint32_t tiles = (n + kScanTile - 1) / kScanTile;
  const size_t counts_bytes = (sizeof(uint32_t) * (size_t)n + 255) / 256 * 256;
  void* scratch = nullptr;
  {
    const bits_status as = pool_alloc(&scratch, counts_bytes + sizeof(uint64_t) * (tiles + 1), st);
    if (as != BITS_OK) return as;
  }
  uint32_t* counts = static_cast<uint32_t*>(scratch);
  auto* part = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + counts_bytes);
  bits_status s = launch_count_search(db, d_a, n, counts, reinterpret_cast<uint64_t*>(part + tiles),
                                      st);
  if (s == BITS_OK) {
    auto* off = reinterpret_cast<unsigned long long*>(d_offsets);
    k_scan_reduce<<<tiles, kScanBlock, 0, st>>>(counts, n, part);
    count_launch();
    k_scan_partials<<<1, 1024, 0, st>>>(part, tiles, off + n);
    count_launch();
    k_scan_down<<<tiles, kScanBlock, 0, st>>>(counts, n, part, off);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_status(e, "enumeration offsets");
  }
  pool_free(scratch, st);
  return s;
}

bits_status run_enumerate_pairs(const bits_db* db, const uint32_t* d_a, uint32_t n,
                                const uint64_t* d_offsets, uint32_t* d_pairs, cudaStream_t st) {
  if (n == 0) return BITS_OK;
  const size_t smem = sizeof(uint32_t) * 2 * top_words(db->lvl.top_size);
  const uint64_t warps_needed = (n + 31) / 32;
  const uint64_t want = (warps_needed + kEnumBlock / 32 - 1) / (kEnumBlock / 32);
  const uint32_t grid = (uint32_t)std::min<uint64_t>(
      want, (uint64_t)enum_blocks_per_sm(smem) * sm_count());
  k_enumerate<<<grid, kEnumBlock, smem, st>>>(
      reinterpret_cast<const uint2*>(d_a), n, db->lvl, db->n, db->enum_e,
      reinterpret_cast<const unsigned long long*>(d_offsets), reinterpret_cast<uint2*>(d_pairs),
      db->err);
  BITS_LAUNCH_CHECK("k_enumerate");
  return BITS_OK;
}

}  // namespace bits
