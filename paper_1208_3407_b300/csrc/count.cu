// bits_count kernels: Algorithm 2's counting loop over Algorithm 1 (ICount).
//
// One thread per query (Sec. "Parallel BITS" assigns one ICount per thread): a coalesced
// 8-byte load of (start, end), the two top-level searches in shared memory,
// the quad-cooperative descent through the 16-ary levels (search.cuh), a
// coalesced 4-byte store of the count, and a block reduction of the 64-bit
// total with one atomic per CTA.
//
// The tree the searches descend is written by levels.cu.
#include "count.cuh"
#include "search.cuh"

namespace bits {
namespace {

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
    quad_descend(L, rs, key_s, re, key_e);
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
