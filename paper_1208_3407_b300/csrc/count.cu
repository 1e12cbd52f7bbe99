// bits_count kernels: Algorithm 2's counting loop over Algorithm 1 (ICount),
// one thread per pair of queries (Sec. 2.4 assigns one ICount per thread;
// two per thread here give four independent searches in flight).
//
// Per thread: one 16-byte load of two (start, end) queries, four searches
// (two ranks per query) through the shared-memory top tree and then through
// the 2^k-element bucket in global memory, one 8-byte store of the two
// counts, and a block reduction of the 64-bit total with one atomic per CTA.
#include "count.cuh"
#include "search.cuh"

namespace bits {
namespace {

constexpr int kCountBlock = 256;

template <bool VEC>
__global__ void __launch_bounds__(kCountBlock)
k_count_search(const uint2* __restrict__ a, uint32_t n, const uint32_t* __restrict__ bs,
               const uint32_t* __restrict__ be, uint32_t nb, const uint32_t* __restrict__ tree,
               int t, int k, uint32_t* __restrict__ counts,
               unsigned long long* __restrict__ total, uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) uint32_t s_tree[];
  __shared__ unsigned long long s_red[32];
  const uint32_t tsz = 1u << t;
  load_tree(s_tree, tree, tsz);
  __syncthreads();

  unsigned long long acc = 0ull;
  bool bad = false;
  const uint32_t npairs = (n >> 1) + (n & 1u);
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs;
       p += gridDim.x * blockDim.x) {
    const bool has1 = 2u * p + 1u < n;
    uint32_t s0, e0, s1 = 0u, e1 = 0u;
    if (VEC && has1) {
      const uint4 q = __ldcs(reinterpret_cast<const uint4*>(a) + p);
      s0 = q.x; e0 = q.y; s1 = q.z; e1 = q.w;
    } else {
      const uint2 q0 = __ldcs(a + 2u * p);
      s0 = q0.x; e0 = q0.y;
      if (has1) {
        const uint2 q1 = __ldcs(a + 2u * p + 1u);
        s1 = q1.x; e1 = q1.y;
      }
    }
    const uint32_t key[4] = {e0, s0 + 1u, e1, s1 + 1u};
    uint32_t pos[4];
    rank_lt_tree<4>(s_tree, tsz, bs, be, nb, k, key, pos);
    uint32_t c0 = icount_from_ranks(pos[0], pos[1], s0, nb);
    uint32_t c1 = icount_from_ranks(pos[2], pos[3], s1, nb);
    if (e0 < s0) { c0 = 0u; bad = true; }
    if (e1 < s1) { c1 = 0u; bad = true; }
    if (!has1) c1 = 0u;
    if (counts) {
      if (VEC && has1) {
        __stcs(reinterpret_cast<uint2*>(counts) + p, make_uint2(c0, c1));
      } else {
        counts[2u * p] = c0;
        if (has1) counts[2u * p + 1u] = c1;
      }
    }
    acc += (unsigned long long)c0 + c1;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_dev_error(err, DEV_ERR_INVALID);
  const unsigned long long sum = block_sum_u64(acc, s_red);
  if (threadIdx.x == 0 && sum) atomicAdd(total, sum);
}

template <bool VEC>
int count_grid(size_t smem) {
  static int per_sm[2] = {0, 0};
  static size_t smem_for[2] = {0, 0};
  const int slot = VEC ? 1 : 0;
  if (per_sm[slot] == 0 || smem_for[slot] != smem) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_count_search<VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_count_search<VEC>, kCountBlock, smem);
    per_sm[slot] = std::max(1, b);
    smem_for[slot] = smem;
  }
  return per_sm[slot];
}

}  // namespace

bits_status launch_count_search(const bits_db* db, const uint32_t* d_a, uint32_t n,
                                uint32_t* d_counts, uint64_t* d_total, cudaStream_t st) {
  BITS_CUDA_TRY(cudaMemsetAsync(d_total, 0, sizeof(uint64_t), st));
  if (n == 0) return BITS_OK;
  const uint32_t tsz = 1u << db->tree_log2;
  const size_t smem = sizeof(uint32_t) * 2 * tsz;
  const bool vec = (reinterpret_cast<uintptr_t>(d_a) % 16 == 0) &&
                   (d_counts == nullptr || reinterpret_cast<uintptr_t>(d_counts) % 8 == 0);
  const uint32_t npairs = (n >> 1) + (n & 1u);
  const uint32_t need = (npairs + kCountBlock - 1) / kCountBlock;
  const uint2* a = reinterpret_cast<const uint2*>(d_a);
  auto* tot = reinterpret_cast<unsigned long long*>(d_total);
  if (vec) {
    const uint32_t grid = std::min<uint32_t>(need, (uint32_t)(count_grid<true>(smem) * sm_count()));
    k_count_search<true><<<grid, kCountBlock, smem, st>>>(a, n, db->bs, db->be, db->n, db->tree,
                                                          db->tree_log2, db->bucket_log2,
                                                          d_counts, tot, db->err);
  } else {
    const uint32_t grid = std::min<uint32_t>(need, (uint32_t)(count_grid<false>(smem) * sm_count()));
    k_count_search<false><<<grid, kCountBlock, smem, st>>>(a, n, db->bs, db->be, db->n, db->tree,
                                                           db->tree_log2, db->bucket_log2,
                                                           d_counts, tot, db->err);
  }
  BITS_LAUNCH_CHECK("k_count_search");
  return BITS_OK;
}

}  // namespace bits
