// bits_count kernels: Algorithm 2's counting loop over Algorithm 1 (ICount).
//
// One thread per query (Sec. "Parallel BITS" assigns one ICount per thread): a coalesced
// 8-byte load of (start, end), the two top-level searches in shared memory,
// the quad-cooperative descent through the 16-ary levels (search.cuh), a
// coalesced 4-byte store of the count, and a block reduction of the 64-bit
// total with one atomic per CTA.
//
// Also here: k_build_levels and k_interleave_level0, which write the
// implicit 16-ary tree of both sorted arrays after the sort, its levels
// stored with node i of the starts and node i of the ends in one 128-byte
// line (search.cuh).
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

struct LevelJob {
  uint32_t* out;
  const uint32_t* src;  // sorted array the level samples
  uint32_t count;       // entries to write (real + padding)
  uint32_t real;        // real entries; the rest are 0xFFFFFFFF
  int shift;            // 4 * level
  int half;             // 0: plain; 1 / 2: the starts' / ends' half of interleaved node pairs
};
struct LevelJobs {
  LevelJob j[2 * (kMaxLevels + kTopRaise + 2)];  // per array: padding, stored levels, top images
};

__global__ void k_build_levels(LevelJobs jobs, uint32_t n) {
  const LevelJob* J = &jobs.j[blockIdx.y];
  uint32_t* out = J->out;
  const uint32_t* src = J->src;
  const uint32_t count = J->count, real = J->real;
  const int shift = J->shift, half = J->half;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    uint32_t v = kU32Max;
    if (i < real) {
      const uint64_t end = min(((uint64_t)i + 1u) << shift, (uint64_t)n);
      v = src[end - 1];
    }
    const uint32_t at = half ? 32u * (i >> 4) + 16u * (uint32_t)(half - 1) + (i & 15u) : i;
    out[at] = v;
  }
}

// Level 0 of both sorted arrays (already padded to 16) into node pairs:
// eight lanes move one 128-byte pair with 16-byte loads and stores.
__global__ void k_interleave_level0(const uint4* __restrict__ bs, const uint4* __restrict__ be,
                                    uint32_t pairs, uint4* __restrict__ out) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < 8u * pairs; t += stride) {
    const uint32_t p = t >> 3, q = t & 7u;
    out[t] = q < 4u ? bs[4u * p + q] : be[4u * p + (q - 4u)];
  }
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

uint32_t round16(uint32_t x) { return (x + 15u) & ~15u; }

void plan_levels(uint32_t n, int top_log2, LevelPlan& p) {
  const uint32_t cap = (1u << top_log2) - 1u;
  p = LevelPlan{};
  p.len[0] = n;
  int J = 0;
  // Past level kMaxTop the top simply grows (at most 1024 entries for n < 2^30).
  while (p.len[J] > cap && J < kMaxTop) {
    p.len[J + 1] = (uint32_t)(((uint64_t)p.len[J] + 15u) / 16u);
    ++J;
  }
  p.J = J;
  // Smaller tops a launch may use: up to kTopRaise levels above J while the
  // level below still spans more than one node.
  int T = J;
  while (T < J + kTopRaise && p.len[T] > 16u) {
    p.len[T + 1] = (uint32_t)(((uint64_t)p.len[T] + 15u) / 16u);
    ++T;
  }
  p.Tmax = T;
  size_t tw = 0;
  for (int t = J; t <= T; ++t) {
    uint32_t ts = 4;
    while (ts < p.len[t] + 1u) ts <<= 1;
    p.top_size_at[t] = ts;
    p.top_off[t] = tw;
    tw += 2 * (size_t)ts;
  }
  p.top_words = tw;
  p.top_size = p.top_size_at[J];
  // words of the stored levels 0 .. Tmax-1, both arrays interleaved by node,
  // each level padded to 16 entries per array
  size_t words = 0;
  for (int j = 0; j < T; ++j) {
    p.off[j] = words;
    words += 2 * (size_t)round16(p.len[j]);
  }
  p.level_words = words;
}

LevelIndex level_view(const bits_db* db, int raise) {
  const LevelPlan& p = db->plan;
  LevelIndex L = db->lvl;
  const int t = std::min(p.J + std::max(raise, 0), p.Tmax);
  L.J = t;
  L.top = db->top + p.top_off[t];
  L.top_size = p.top_size_at[t];
  return L;
}

bits_status build_levels(bits_db* db, cudaStream_t st) {
  const LevelPlan& p = db->plan;
  LevelIndex& L = db->lvl;
  L = LevelIndex{};
  L.J = p.J;
  L.top_size = p.top_size;
  L.top = db->top + p.top_off[p.J];
  for (int j = 0; j <= p.Tmax; ++j) L.len[j] = p.len[j];
  L.x[0] = db->bs;
  L.x[1] = db->be;
  for (int j = 0; j < p.Tmax; ++j) L.il[j] = db->levels + p.off[j];
  LevelJobs jobs{};
  int nj = 0;
  for (int a = 0; a < 2; ++a) {
    uint32_t* X = a ? db->be : db->bs;
    // padding of the plain sorted array
    jobs.j[nj++] = LevelJob{X + db->n, X, round16(db->n) - db->n, 0u, 0, 0};
    for (int j = 1; j < p.Tmax; ++j)
      jobs.j[nj++] = LevelJob{db->levels + p.off[j], X, round16(p.len[j]), p.len[j], 4 * j, a + 1};
    for (int t = p.J; t <= p.Tmax; ++t)
      jobs.j[nj++] = LevelJob{db->top + p.top_off[t] + (size_t)a * p.top_size_at[t], X,
                              p.top_size_at[t], p.len[t], 4 * t, 0};
  }
  uint32_t biggest = 1;
  for (int k = 0; k < nj; ++k) biggest = std::max(biggest, jobs.j[k].count);
  const dim3 grid(std::min<uint32_t>((biggest + 255) / 256, 4096), nj);
  k_build_levels<<<grid, 256, 0, st>>>(jobs, db->n);
  BITS_LAUNCH_CHECK("k_build_levels");
  if (p.Tmax > 0) {
    // Runs after the padding of the plain arrays above (stream order).
    const uint32_t pairs = round16(db->n) / 16u;
    const uint32_t blocks =
        std::min<uint32_t>((8u * pairs + 255u) / 256u, (uint32_t)(sm_count() * 8));
    k_interleave_level0<<<blocks, 256, 0, st>>>(reinterpret_cast<const uint4*>(db->bs),
                                                reinterpret_cast<const uint4*>(db->be), pairs,
                                                reinterpret_cast<uint4*>(db->levels + p.off[0]));
    BITS_LAUNCH_CHECK("k_interleave_level0");
  }
  return BITS_OK;
}

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
