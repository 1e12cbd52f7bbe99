// Learned index (two-stage RMI, Kraska et al. 2018) over each sorted array:
// on-device fitting, and bits_count through it.
//
// Fitting, all on the device after the sort.  Both stages are least-squares
// lines of rank against key; their sums are exact integers (the part's fp64
// rate is a small fraction of its integer rate, and exact sums lose nothing
// to cancellation):
//   1. k_rmi_chunk_moments: per chunk of kChunk consecutive ranks i (one
//      warp each), the sums of X_i, X_i^2 and i * X_i (64- and 128-bit
//      integers).
//   2. k_rmi_scan_block, twice: exclusive prefix of those sums, first within
//      each group of 1024 chunks, then over the groups, with the whole
//      array's sums at the end.  The host fits the root from the
//      whole-array sums and rounds it to fp32 (slope clamped to >= 0 so the
//      root is monotone).
//   3. k_rmi_bounds: the slice [lo, hi) of ranks every leaf owns, by a
//      binary search per leaf boundary (the root is monotone, so the leaf of
//      X_i never decreases with i).
//   4. k_rmi_boundary_moments: the prefix sums at every slice boundary (the
//      group and chunk prefixes plus the ranks of the boundary's chunk below
//      it).
//   5. k_rmi_fit: a leaf's sums are differences of its two boundaries'
//      prefixes; from them, exactly in 128-bit integers, the moments of
//      (key - base, rank - lo), and the fp32 slope (>= 0) and intercept.
//   6. k_rmi_errors: with the search's own rmi_predict, the smallest and
//      largest (true rank - prediction) over every key of the slice (and one
//      past each key), so that every query routed to the leaf has its rank in
//      [prediction + err_lo, prediction + err_hi].
#include <cmath>

#include "count.cuh"
#include "rmi.cuh"
#include "rmi_search.cuh"

namespace bits {
namespace {

using u64 = unsigned long long;
using u128 = unsigned __int128;
using i128 = __int128;

constexpr int kRmiBlock = 256;
constexpr uint32_t kChunk = 1024;  // ranks per chunk of the moment prefix sums
constexpr int kScanThreads = 1024;

// Sums over a run of ranks i of the sorted array X.
struct Moments {
  u64 s1;   // sum of X_i             (< 2^62 for n < 2^30)
  u128 s2;  // sum of X_i^2           (< 2^94)
  u128 s3;  // sum of i * X_i         (< 2^92)
};

// Moments of a run stored as three arrays (16-byte aligned for the 128-bit ones).
struct MomentArrays {
  u64* s1;
  u128* s2;
  u128* s3;
};

__device__ __forceinline__ void add_key(Moments& m, uint32_t i, uint32_t x) {
  m.s1 += x;
  m.s2 += (u128)((u64)x * x);
  m.s3 += (u128)((u64)i * x);
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int o) {
  const u64 lo = __shfl_xor_sync(0xFFFFFFFFu, (u64)v, o);
  const u64 hi = __shfl_xor_sync(0xFFFFFFFFu, (u64)(v >> 64), o);
  return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ Moments warp_sum_moments(Moments m) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m.s1 += __shfl_xor_sync(0xFFFFFFFFu, m.s1, o);
    m.s2 += shfl_xor_u128(m.s2, o);
    m.s3 += shfl_xor_u128(m.s3, o);
  }
  return m;
}

__device__ __forceinline__ void store_moments(const MomentArrays& A, size_t k, const Moments& m) {
  A.s1[k] = m.s1;
  A.s2[k] = m.s2;
  A.s3[k] = m.s3;
}

__device__ __forceinline__ Moments load_moments(const MomentArrays& A, size_t k) {
  return Moments{A.s1[k], A.s2[k], A.s3[k]};
}

// The nearest double to an exact 128-bit integer (two roundings at most).
__device__ __forceinline__ double i128_to_double(i128 v) {
  const bool neg = v < 0;
  const u128 u = neg ? (u128)(-v) : (u128)v;
  const double d = (double)(u64)(u >> 64) * 18446744073709551616.0 + (double)(u64)u;
  return neg ? -d : d;
}

// One warp per chunk: lane j adds ranks chunk * kChunk + j + 32 k.
__global__ void __launch_bounds__(kRmiBlock)
k_rmi_chunk_moments(const uint32_t* __restrict__ X, uint32_t n, uint32_t nchunks,
                    MomentArrays chunks) {
  const uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= nchunks) return;
  const uint32_t base = c * kChunk;
  Moments m{0ull, 0, 0};
  if (base + kChunk <= n) {
    #pragma unroll 8
    for (uint32_t k = 0; k < kChunk / 32; ++k) {
      const uint32_t i = base + k * 32 + lane_id();
      add_key(m, i, __ldcs(X + i));
    }
  } else {
    for (uint32_t i = base + lane_id(); i < n; i += 32) add_key(m, i, X[i]);
  }
  m = warp_sum_moments(m);
  if (lane_id() == 0) store_moments(chunks, c, m);
}

// Items [b * 1024, min(count, (b + 1) * 1024)) of CTA b become exclusive
// prefixes (within the CTA's group) in place; the group's total goes to
// totals[b].
__global__ void __launch_bounds__(kScanThreads)
k_rmi_scan_block(MomentArrays items, uint32_t count, MomentArrays totals) {
  __shared__ Moments s_w[kScanThreads / 32];
  const uint32_t k = blockIdx.x * kScanThreads + threadIdx.x;
  const Moments own = k < count ? load_moments(items, k) : Moments{0ull, 0, 0};
  const unsigned lane = lane_id(), w = threadIdx.x >> 5;
  Moments inc = own;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 a1 = __shfl_up_sync(0xFFFFFFFFu, inc.s1, o);
    const u64 a2l = __shfl_up_sync(0xFFFFFFFFu, (u64)inc.s2, o);
    const u64 a2h = __shfl_up_sync(0xFFFFFFFFu, (u64)(inc.s2 >> 64), o);
    const u64 a3l = __shfl_up_sync(0xFFFFFFFFu, (u64)inc.s3, o);
    const u64 a3h = __shfl_up_sync(0xFFFFFFFFu, (u64)(inc.s3 >> 64), o);
    if (lane >= (unsigned)o) {
      inc.s1 += a1;
      inc.s2 += ((u128)a2h << 64) | a2l;
      inc.s3 += ((u128)a3h << 64) | a3l;
    }
  }
  if (lane == 31) s_w[w] = inc;
  __syncthreads();
  Moments run{0ull, 0, 0};
  for (unsigned v = 0; v < w; ++v) {
    run.s1 += s_w[v].s1;
    run.s2 += s_w[v].s2;
    run.s3 += s_w[v].s3;
  }
  run.s1 += inc.s1 - own.s1;
  run.s2 += inc.s2 - own.s2;
  run.s3 += inc.s3 - own.s3;
  if (k < count) store_moments(items, k, run);
  if (threadIdx.x == kScanThreads - 1) {
    run.s1 += own.s1;
    run.s2 += own.s2;
    run.s3 += own.s3;
    store_moments(totals, blockIdx.x, run);
  }
}

// lo[l] = the first rank whose key the root sends to leaf l or above (n if
// none): a binary search per boundary l in [0, nleaves].
__global__ void k_rmi_bounds(const uint32_t* __restrict__ X, uint32_t n, float ra, float rb,
                             uint32_t nleaves, uint32_t* __restrict__ lo_out) {
  const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l > nleaves) return;
  uint32_t lo = 0, hi = n;  // the answer lies in [lo, hi]
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (rmi_root(ra, rb, X[mid], nleaves) >= l) hi = mid;
    else lo = mid + 1;
  }
  lo_out[l] = lo;
}

// One warp per slice boundary l in [0, nleaves]: the moment prefix at rank
// p = lo[l] (sums over ranks [0, p)) = the prefix of the group of p's chunk
// + the prefix of the chunk within its group + the ranks of the chunk below
// p.  A boundary at p = n with n a multiple of kChunk takes the last chunk
// whole (n >= 1 here).
__global__ void __launch_bounds__(kRmiBlock)
k_rmi_boundary_moments(const uint32_t* __restrict__ X, const uint32_t* __restrict__ lo,
                       uint32_t nleaves, uint32_t nchunks, MomentArrays chunks,
                       MomentArrays groups, MomentArrays at) {
  const uint32_t l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (l > nleaves) return;
  const uint32_t p = lo[l], c = min(p / kChunk, nchunks - 1);
  Moments m{0ull, 0, 0};
  for (uint32_t i = c * kChunk + lane_id(); i < p; i += 32) add_key(m, i, X[i]);
  m = warp_sum_moments(m);
  if (lane_id() == 0) {
    const Moments g = load_moments(groups, c / kScanThreads), pre = load_moments(chunks, c);
    m.s1 += g.s1 + pre.s1;
    m.s2 += g.s2 + pre.s2;
    m.s3 += g.s3 + pre.s3;
    store_moments(at, l, m);
  }
}

__global__ void k_rmi_fit(const uint32_t* __restrict__ X, uint32_t n,
                          const uint32_t* __restrict__ lo, MomentArrays at, uint32_t nleaves,
                          bits_rmi_leaf* __restrict__ leaves) {
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < nleaves;
       l += gridDim.x * blockDim.x) {
    const uint32_t first = lo[l], last = lo[l + 1], cnt = last - first;
    uint32_t base = 0;
    if (first < n) base = X[first];
    else if (n) base = X[n - 1];
    double slope = 0.0, icpt = 0.0;
    if (cnt >= 2) {
      // Sums over the slice of X_i, X_i^2, i * X_i, then of x = X_i - base
      // and y = i - first (all exact):
      //   Sx  = S1 - c base            Sy  = c (c - 1) / 2
      //   Sxx = S2 - 2 base S1 + c base^2
      //   Sxy = S3 - first S1 - base c (c - 1) / 2
      const Moments hi = load_moments(at, l + 1), lw = load_moments(at, l);
      const i128 c = cnt, bs = base, f = first;
      const i128 s1 = (i128)(hi.s1 - lw.s1), s2 = (i128)(hi.s2 - lw.s2),
                 s3 = (i128)(hi.s3 - lw.s3);
      const i128 tri = c * (c - 1) / 2;
      const i128 sx = s1 - c * bs, sy = tri;
      const i128 sxx = s2 - 2 * bs * s1 + c * bs * bs;
      const i128 sxy = s3 - f * s1 - bs * tri;
      const i128 den = c * sxx - sx * sx, num = c * sxy - sx * sy;
      if (den > 0) slope = i128_to_double(num) / i128_to_double(den);
      if (!(slope > 0.0)) slope = 0.0;
      icpt = (i128_to_double(sy) - slope * i128_to_double(sx)) / (double)cnt;
    }
    bits_rmi_leaf lf;
    lf.base_key = base;
    lf.lo = first;
    lf.slope = (float)slope;
    lf.icpt = (float)icpt;
    lf.err_lo = 0;
    lf.err_hi = 0;
    lf.hi = last;
    lf.pad = 0;
    leaves[l] = lf;
  }
}

// Each thread takes kErrKeys consecutive ranks (usually all in one leaf): it
// folds their errors per leaf run, sends any run that ends inside its ranks
// straight to the leaf with atomics, and the run it ends on is combined with
// the other lanes' last runs of the same leaf before one lane sends it.
constexpr uint32_t kErrKeys = 8;

__device__ __forceinline__ void send_errors(bits_rmi_leaf* leaves, uint32_t l, int mn, int mx) {
  if (mn < 0) atomicMin(&leaves[l].err_lo, mn);
  if (mx > 0) atomicMax(&leaves[l].err_hi, mx);
}

__global__ void __launch_bounds__(kRmiBlock)
k_rmi_errors(const uint32_t* __restrict__ X, uint32_t n, float ra, float rb, uint32_t nleaves,
             bits_rmi_leaf* __restrict__ leaves) {
  const uint32_t i0 = (blockIdx.x * blockDim.x + threadIdx.x) * kErrKeys;
  uint32_t l = 0xFFFFFFFFu;  // leaf of the current run (none yet)
  int e_lo = 0x7FFFFFFF, e_hi = -0x7FFFFFFF;
  if (i0 < n) {
    uint32_t key[kErrKeys];
    const uint32_t m = min(kErrKeys, n - i0);
    if (m == kErrKeys && (reinterpret_cast<uintptr_t>(X + i0) & 15u) == 0) {
      const uint4 v0 = __ldcs(reinterpret_cast<const uint4*>(X + i0));
      const uint4 v1 = __ldcs(reinterpret_cast<const uint4*>(X + i0) + 1);
      key[0] = v0.x; key[1] = v0.y; key[2] = v0.z; key[3] = v0.w;
      key[4] = v1.x; key[5] = v1.y; key[6] = v1.z; key[7] = v1.w;
    } else {
      #pragma unroll
      for (uint32_t j = 0; j < kErrKeys; ++j) key[j] = j < m ? X[i0 + j] : 0u;
    }
    uint32_t prev = i0 > 0 ? X[i0 - 1] : 0u;
    float slope = 0.f, icpt = 0.f;
    uint32_t base = 0, lo = 0, cnt = 0;
    #pragma unroll
    for (uint32_t j = 0; j < kErrKeys; ++j) {
      if (j < m) {
        const uint32_t i = i0 + j, k = key[j];
        const uint32_t lk = rmi_root(ra, rb, k, nleaves);
        if (lk != l) {
          if (l != 0xFFFFFFFFu) send_errors(leaves, l, e_lo, e_hi);
          l = lk;
          const bits_rmi_leaf lf = leaves[l];
          slope = lf.slope;
          icpt = lf.icpt;
          base = lf.base_key;
          lo = lf.lo;
          cnt = lf.hi - lf.lo;
          e_lo = 0x7FFFFFFF;
          e_hi = -0x7FFFFFFF;
        }
        const int p = rmi_predict(slope, icpt, base, cnt, k);
        const int local = (int)(i - lo);
        e_hi = max(e_hi, local + 1 - p);  // a query just above k has rank i + 1
        if (i == lo || prev != k) e_lo = min(e_lo, local - p);  // rank of k itself
        prev = k;
      }
    }
  }
  // Lanes hold consecutive ranks, so the lanes that end on one leaf are a
  // contiguous run: from this lane's run head up to the next head.
  const unsigned lane = lane_id();
  const uint32_t prev_l = __shfl_up_sync(0xFFFFFFFFu, l, 1);
  const unsigned heads = __ballot_sync(0xFFFFFFFFu, lane == 0 || prev_l != l);
  const unsigned below = heads & (0xFFFFFFFFu >> (31 - lane));  // heads at or below this lane
  const unsigned above = heads & ~(0xFFFFFFFFu >> (31 - lane));  // heads above this lane
  const int first_lane = 31 - __clz(below);
  const unsigned end_mask = above ? (above & (0u - above)) - 1u : 0xFFFFFFFFu;
  const unsigned peers = end_mask & ~((1u << first_lane) - 1u);
  const int mn = __reduce_min_sync(peers, e_lo);
  const int mx = __reduce_max_sync(peers, e_hi);
  if (l != 0xFFFFFFFFu && (int)lane == first_lane) send_errors(leaves, l, mn, mx);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_count_rmi(const uint2* __restrict__ a, uint32_t n, LevelIndex L, RmiView R, uint32_t nb,
            uint32_t* __restrict__ counts, unsigned long long* __restrict__ total,
            uint32_t* __restrict__ err) {
  __shared__ unsigned long long s_red[32];
  unsigned long long acc = 0ull;
  bool bad = false;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const uint32_t i = base + threadIdx.x;
    const bool valid = i < n;
    uint2 q = make_uint2(0u, 0u);
    if (valid) q = __ldcs(a + i);
    uint32_t rs, re;
    rmi_rank2(R, L, nb, q.y, q.x + 1u, rs, re);
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
  grid_dependency_wait();  // the total was zeroed by the kernel before this one
  if (threadIdx.x == 0 && sum) atomicAdd(total, sum);
}

template <int BLOCK>
bits_status launch_rmi(const bits_db* db, const uint2* a, uint32_t n, uint32_t* d_counts,
                       uint64_t* d_total, cudaStream_t st) {
  const int per_sm =
      kernel_blocks_per_sm(reinterpret_cast<const void*>(k_count_rmi<BLOCK>), BLOCK, 0);
  const uint32_t need = (n + BLOCK - 1) / BLOCK;
  const uint32_t grid = std::min<uint32_t>(need, (uint32_t)(per_sm * sm_count()));
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  pdl_config(cfg, attr, dim3(grid), dim3(BLOCK), 0, st);
  BITS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_count_rmi<BLOCK>, a, n, db->lvl, rmi_view(db), db->n,
                                   d_counts, reinterpret_cast<unsigned long long*>(d_total),
                                   db->err));
  BITS_LAUNCH_CHECK("k_count_rmi");
  return BITS_OK;
}

}  // namespace

RmiView rmi_view(const bits_db* db) {
  RmiView R{};
  for (int a = 0; a < 2; ++a) {
    R.leaves[a] = db->rmi[a].leaves;
    R.ra[a] = db->rmi[a].root_slope;
    R.rb[a] = db->rmi[a].root_icpt;
  }
  R.nleaves = 1u << db->rmi[0].leaves_log2;
  return R;
}

bits_status rmi_build(const uint32_t* X, uint32_t n, bits_rmi& rmi, cudaStream_t st) {
  const uint32_t L = 1u << rmi.leaves_log2;
  const uint32_t nchunks = (n + kChunk - 1) / kChunk;
  const uint32_t ngroups = (nchunks + kScanThreads - 1) / kScanThreads;  // <= 1024 (n < 2^30)
  // Scratch: chunk moments [nchunks] | group moments [ngroups + 1] |
  // boundary moments [L + 1] | lo [L + 1].
  auto arrays_bytes = [](size_t m) {
    return (sizeof(u64) * m + 255) / 256 * 256 + 2 * ((sizeof(u128) * m + 255) / 256 * 256);
  };
  const size_t chunk_bytes = arrays_bytes((size_t)nchunks + 1);
  const size_t group_bytes = arrays_bytes((size_t)ngroups + 1);
  const size_t at_bytes = arrays_bytes((size_t)L + 1);
  const size_t bytes = chunk_bytes + group_bytes + at_bytes + sizeof(uint32_t) * ((size_t)L + 1);
  void* scratch = nullptr;
  {
    const bits_status as = pool_alloc(&scratch, bytes, st);
    if (as != BITS_OK) return as;
  }
  auto carve = [](char* p, size_t m) {
    MomentArrays A;
    A.s1 = reinterpret_cast<u64*>(p);
    p += (sizeof(u64) * m + 255) / 256 * 256;
    A.s2 = reinterpret_cast<u128*>(p);
    p += (sizeof(u128) * m + 255) / 256 * 256;
    A.s3 = reinterpret_cast<u128*>(p);
    return A;
  };
  char* base = static_cast<char*>(scratch);
  const MomentArrays chunks = carve(base, (size_t)nchunks + 1);
  const MomentArrays groups = carve(base + chunk_bytes, (size_t)ngroups + 1);
  const MomentArrays at = carve(base + chunk_bytes + group_bytes, (size_t)L + 1);
  uint32_t* lo = reinterpret_cast<uint32_t*>(base + chunk_bytes + group_bytes + at_bytes);
  auto done = [&](bits_status s) {
    pool_free(scratch, st);
    return s;
  };
  if (cudaMemsetAsync(scratch, 0, bytes, st) != cudaSuccess)
    return done(cuda_status(cudaGetLastError(), "cudaMemsetAsync(rmi scratch)"));

  if (n) {
    const uint32_t warps_per_block = kRmiBlock / 32;
    k_rmi_chunk_moments<<<(nchunks + warps_per_block - 1) / warps_per_block, kRmiBlock, 0, st>>>(
        X, n, nchunks, chunks);
    count_launch();
    k_rmi_scan_block<<<ngroups, kScanThreads, 0, st>>>(chunks, nchunks, groups);
    count_launch();
    MomentArrays grand = groups;  // entry ngroups: the whole array
    grand.s1 += ngroups;
    grand.s2 += ngroups;
    grand.s3 += ngroups;
    k_rmi_scan_block<<<1, kScanThreads, 0, st>>>(groups, ngroups, grand);
    count_launch();
  }

  // Root: least-squares line of t = i * L / n against the key over the
  // whole array, from its exact sums (host 128-bit integers):
  //   slope_i = (n Sxi - Sx Si) / (n Sxx - Sx^2),  Si = n (n - 1) / 2.
  float ra = 0.f, rb = 0.f;
  if (n >= 2) {
    u64 h1 = 0;
    u128 h2 = 0, h3 = 0;
    if (cudaMemcpyAsync(&h1, groups.s1 + ngroups, sizeof(h1), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(&h2, groups.s2 + ngroups, sizeof(h2), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(&h3, groups.s3 + ngroups, sizeof(h3), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return done(cuda_status(cudaGetLastError(), "rmi root sums"));
    const i128 c = n, sx = (i128)h1, sxx = (i128)h2, sxi = (i128)h3;
    const i128 si = c * (c - 1) / 2;
    const i128 den = c * sxx - sx * sx, num = c * sxi - sx * si;
    const double scale = (double)L / (double)n;
    double a = den > 0 ? (double)num / (double)den * scale : 0.0;
    if (!(a > 0.0) || !std::isfinite(a)) a = 0.0;
    // Intercept through the means: mean t = scale (n - 1) / 2, mean key = Sx / n.
    const double b = scale * (double)(n - 1) / 2.0 - a * ((double)h1 / (double)n);
    ra = (float)a;
    rb = (float)b;
    if (!std::isfinite(rb)) {
      ra = 0.f;
      rb = 0.f;
    }
  }
  rmi.root_slope = ra;
  rmi.root_icpt = rb;

  k_rmi_bounds<<<(L + 1 + 255) / 256, 256, 0, st>>>(X, n, ra, rb, L, lo);
  count_launch();
  if (n) {
    k_rmi_boundary_moments<<<((L + 1) * 32u + kRmiBlock - 1) / kRmiBlock, kRmiBlock, 0, st>>>(
        X, lo, L, nchunks, chunks, groups, at);
    count_launch();
  }
  k_rmi_fit<<<(L + 255) / 256, 256, 0, st>>>(X, n, lo, at, L, rmi.leaves);
  count_launch();
  if (n) {
    const uint32_t threads = (n + kErrKeys - 1) / kErrKeys;
    k_rmi_errors<<<(threads + kRmiBlock - 1) / kRmiBlock, kRmiBlock, 0, st>>>(X, n, ra, rb, L,
                                                                            rmi.leaves);
    count_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return done(cuda_status(e, "rmi build kernels"));
  return done(BITS_OK);
}

bits_status launch_count_rmi(const bits_db* db, const uint32_t* d_a, uint32_t n,
                             uint32_t* d_counts, uint64_t* d_total, cudaStream_t st,
                             const TuneCount* tc) {
  bits_status s = launch_zero_total(d_total, st);
  if (s != BITS_OK || n == 0) return s;
  const int block = tc ? tc->block : count_params(db, BITS_METHOD_RMI, n, d_counts != nullptr).block;
  const uint2* a = reinterpret_cast<const uint2*>(d_a);
  return block == 512 ? launch_rmi<512>(db, a, n, d_counts, d_total, st)
                      : launch_rmi<256>(db, a, n, d_counts, d_total, st);
}

}  // namespace bits
