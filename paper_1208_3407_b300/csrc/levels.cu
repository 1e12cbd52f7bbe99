// The implicit 16-ary tree of both sorted arrays (search.cuh), written after
// the database sort: the level plan (which levels are stored, which serves
// as the shared-memory top), the padding of the sorted arrays, every stored
// level with node i of the starts and node i of the ends in one 128-byte
// line, and the top images the searches copy to shared memory.
#include "count.cuh"
#include "search.cuh"

namespace bits {
namespace {

struct LevelJob {
  uint32_t* out;
  const uint32_t* src;  // sorted array the level samples
  uint32_t begin;       // first entry to write (level 1's real entries come with level 0)
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
  for (uint32_t i = J->begin + blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += gridDim.x * blockDim.x) {
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
// eight lanes move one 128-byte pair with 16-byte loads and stores.  When
// level 1 is stored (l1 != nullptr), the lanes holding the last four keys of
// a node also write its level-1 entry, the node's last real key, into
// level 1's node pairs, so that level 1 costs no second read of the arrays.
__global__ void k_interleave_level0(const uint4* __restrict__ bs, const uint4* __restrict__ be,
                                    uint32_t pairs, uint32_t n, uint4* __restrict__ out,
                                    uint32_t* __restrict__ l1) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < 8u * pairs; t += stride) {
    const uint32_t p = t >> 3, q = t & 7u;
    const uint4 v = q < 4u ? bs[4u * p + q] : be[4u * p + (q - 4u)];
    out[t] = v;
    if (l1 && (q & 3u) == 3u) {
      const uint32_t* x = reinterpret_cast<const uint32_t*>(q < 4u ? bs : be);
      const uint32_t last = 16u * p + 15u < n ? v.w : x[n - 1u];
      l1[32u * (p >> 4) + 16u * (q >> 2) + (p & 15u)] = last;
    }
  }
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
    jobs.j[nj++] = LevelJob{X + db->n, X, 0u, round16(db->n) - db->n, 0u, 0, 0};
    // Level 1's real entries are written with level 0's node pairs below.
    for (int j = 1; j < p.Tmax; ++j)
      jobs.j[nj++] = LevelJob{db->levels + p.off[j], X, j == 1 ? p.len[1] : 0u, round16(p.len[j]),
                              p.len[j], 4 * j, a + 1};
    for (int t = p.J; t <= p.Tmax; ++t)
      jobs.j[nj++] = LevelJob{db->top + p.top_off[t] + (size_t)a * p.top_size_at[t], X, 0u,
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
    k_interleave_level0<<<blocks, 256, 0, st>>>(
        reinterpret_cast<const uint4*>(db->bs), reinterpret_cast<const uint4*>(db->be), pairs,
        db->n, reinterpret_cast<uint4*>(db->levels + p.off[0]),
        p.Tmax > 1 ? db->levels + p.off[1] : nullptr);
    BITS_LAUNCH_CHECK("k_interleave_level0");
  }
  return BITS_OK;
}

}  // namespace bits
