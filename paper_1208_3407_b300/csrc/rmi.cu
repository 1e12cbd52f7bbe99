// Learned index (two-stage RMI, Kraska et al. 2018) over each sorted array:
// on-device fitting, and bits_count through it.
//
// Fitting, all on the device after the sort:
//   1. k_rmi_root_sums: least-squares sums (fp64) of the key against the
//      target leaf position i * 2^L / n; the host turns them into the fp32
//      root (slope, intercept), slope clamped to >= 0 so the root is monotone.
//   2. k_rmi_bounds: the slice [lo, hi) of ranks every leaf owns (contiguous
//      because the root is monotone).
//   3. k_rmi_leaf_sums: per-leaf least-squares sums (fp64) of rank-in-slice
//      against key - base, reduced by warp segments, one atomic per leaf run.
//   4. k_rmi_fit: per-leaf fp32 slope (>= 0) and intercept.
//   5. k_rmi_errors: with the search's own rmi_predict, the smallest and
//      largest (true rank - prediction) over every key of the slice (and one
//      past each key), so that every query routed to the leaf has its rank in
//      [prediction + err_lo, prediction + err_hi].
#include <cmath>

#include "count.cuh"
#include "rmi.cuh"
#include "rmi_search.cuh"

namespace bits {
namespace {

constexpr int kRmiBlock = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__global__ void __launch_bounds__(kRmiBlock)
k_rmi_root_sums(const uint32_t* __restrict__ X, uint32_t n, double t_per_rank,
                double* __restrict__ sums) {
  __shared__ double s_red[4][kRmiBlock / 32];
  const uint32_t x0 = X[0];
  double sx = 0, st = 0, sxx = 0, sxt = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double x = (double)(X[i] - x0), t = (double)i * t_per_rank;
    sx += x;
    st += t;
    sxx = fma(x, x, sxx);
    sxt = fma(x, t, sxt);
  }
  sx = warp_sum_d(sx);
  st = warp_sum_d(st);
  sxx = warp_sum_d(sxx);
  sxt = warp_sum_d(sxt);
  const unsigned w = threadIdx.x >> 5;
  if (lane_id() == 0) {
    s_red[0][w] = sx;
    s_red[1][w] = st;
    s_red[2][w] = sxx;
    s_red[3][w] = sxt;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0;
    for (int k = 0; k < kRmiBlock / 32; ++k) v += s_red[threadIdx.x][k];
    atomicAdd(sums + threadIdx.x, v);
  }
}

__global__ void k_rmi_bounds(const uint32_t* __restrict__ X, uint32_t n, float ra, float rb,
                             uint32_t nleaves, uint32_t* __restrict__ lo_out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
    const int prev = i == 0 ? -1 : (int)rmi_root(ra, rb, X[i - 1], nleaves);
    const int cur = i == n ? (int)nleaves : (int)rmi_root(ra, rb, X[i], nleaves);
    for (int l = prev + 1; l <= cur; ++l) lo_out[l] = i;
  }
}

__global__ void __launch_bounds__(kRmiBlock)
k_rmi_leaf_sums(const uint32_t* __restrict__ X, uint32_t n, float ra, float rb, uint32_t nleaves,
                const uint32_t* __restrict__ lo, double* __restrict__ sums) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned lane = lane_id();
  const bool valid = i < n;
  uint32_t l = 0xFFFFFFFFu;
  double v[4] = {0, 0, 0, 0};
  if (valid) {
    const uint32_t key = X[i];
    l = rmi_root(ra, rb, key, nleaves);
    const uint32_t first = lo[l];
    const double x = (double)(key - X[first]), y = (double)(i - first);
    v[0] = x;
    v[1] = y;
    v[2] = x * x;
    v[3] = x * y;
  }
  // Segmented reduction: lanes of one leaf are contiguous (X sorted, root monotone).
  #pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t ol = __shfl_down_sync(0xFFFFFFFFu, l, off);
    #pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double ov = __shfl_down_sync(0xFFFFFFFFu, v[k], off);
      if (lane + off < 32 && ol == l) v[k] += ov;
    }
  }
  const uint32_t pl = __shfl_up_sync(0xFFFFFFFFu, l, 1);
  if (valid && (lane == 0 || pl != l)) {
    #pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(sums + 4 * (size_t)l + k, v[k]);
  }
}

__global__ void k_rmi_fit(const uint32_t* __restrict__ X, uint32_t n,
                          const uint32_t* __restrict__ lo, const double* __restrict__ sums,
                          uint32_t nleaves, bits_rmi_leaf* __restrict__ leaves) {
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < nleaves;
       l += gridDim.x * blockDim.x) {
    const uint32_t first = lo[l], last = lo[l + 1], cnt = last - first;
    uint32_t base = 0;
    if (first < n) base = X[first];
    else if (n) base = X[n - 1];
    double slope = 0.0, icpt = 0.0;
    if (cnt >= 2) {
      const double c = (double)cnt;
      const double mx = sums[4 * (size_t)l] / c, my = sums[4 * (size_t)l + 1] / c;
      const double vxx = sums[4 * (size_t)l + 2] / c - mx * mx;
      const double cxy = sums[4 * (size_t)l + 3] / c - mx * my;
      if (vxx > 0.0) slope = cxy / vxx;
      if (!(slope > 0.0)) slope = 0.0;
      icpt = my - slope * mx;
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

__global__ void __launch_bounds__(kRmiBlock)
k_rmi_errors(const uint32_t* __restrict__ X, uint32_t n, float ra, float rb, uint32_t nleaves,
             bits_rmi_leaf* __restrict__ leaves) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < n;
  uint32_t l = 0xFFFFFFFFu;
  int e_lo = 0x7FFFFFFF, e_hi = -0x7FFFFFFF;
  if (valid) {
    const uint32_t key = X[i];
    l = rmi_root(ra, rb, key, nleaves);
    const bits_rmi_leaf lf = leaves[l];
    const uint32_t cnt = lf.hi - lf.lo;
    const int p = rmi_predict(lf.slope, lf.icpt, lf.base_key, cnt, key);
    const int local = (int)(i - lf.lo);
    e_hi = local + 1 - p;  // a query just above key has rank i + 1
    if (i == lf.lo || X[i - 1] != key) e_lo = local - p;  // rank of key itself
  }
  const unsigned peers = __match_any_sync(0xFFFFFFFFu, l);
  const int mn = __reduce_min_sync(peers, e_lo);
  const int mx = __reduce_max_sync(peers, e_hi);
  if (valid && (int)lane_id() == __ffs(peers) - 1) {
    if (mn < 0) atomicMin(&leaves[l].err_lo, mn);
    if (mx > 0) atomicMax(&leaves[l].err_hi, mx);
  }
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
  // scratch: 4 root sums | lo[L + 1] | leaf sums [L][4]
  const size_t off_lo = 256;
  const size_t off_sums = (off_lo + sizeof(uint32_t) * (L + 1) + 255) / 256 * 256;
  const size_t bytes = off_sums + sizeof(double) * 4 * (size_t)L;
  void* scratch = nullptr;
  {
    const bits_status as = pool_alloc(&scratch, bytes, st);
    if (as != BITS_OK) return as;
  }
  double* root_sums = static_cast<double*>(scratch);
  uint32_t* lo = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch) + off_lo);
  double* leaf_sums = reinterpret_cast<double*>(static_cast<char*>(scratch) + off_sums);
  auto done = [&](bits_status s) {
    pool_free(scratch, st);
    return s;
  };
  if (cudaMemsetAsync(scratch, 0, bytes, st) != cudaSuccess)
    return done(cuda_status(cudaGetLastError(), "cudaMemsetAsync(rmi scratch)"));

  float ra = 0.f, rb = 0.f;
  if (n >= 2) {
    const int grid = std::max(1, std::min<int>(sm_count() * 8, (n + kRmiBlock - 1) / kRmiBlock));
    k_rmi_root_sums<<<grid, kRmiBlock, 0, st>>>(X, n, (double)L / (double)n, root_sums);
    count_launch();
    double h[4] = {0, 0, 0, 0};
    uint32_t x0 = 0;
    if (cudaMemcpyAsync(h, root_sums, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&x0, X, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return done(cuda_status(cudaGetLastError(), "rmi root sums"));
    const double c = (double)n;
    const double den = c * h[2] - h[0] * h[0];
    double a = den > 0 ? (c * h[3] - h[0] * h[1]) / den : 0.0;
    if (!(a > 0.0) || !std::isfinite(a)) a = 0.0;
    const double b = (h[1] - a * h[0]) / c;
    ra = (float)a;
    rb = (float)(b - a * (double)x0);
    if (!std::isfinite(rb)) {
      ra = 0.f;
      rb = 0.f;
    }
  }
  rmi.root_slope = ra;
  rmi.root_icpt = rb;

  const int gb = std::max(1, std::min<int>(sm_count() * 8, (n + 1 + 255) / 256));
  k_rmi_bounds<<<gb, 256, 0, st>>>(X, n, ra, rb, L, lo);
  count_launch();
  if (n) {
    const uint32_t blocks = (n + kRmiBlock - 1) / kRmiBlock;
    k_rmi_leaf_sums<<<blocks, kRmiBlock, 0, st>>>(X, n, ra, rb, L, lo, leaf_sums);
    count_launch();
  }
  k_rmi_fit<<<(L + 255) / 256, 256, 0, st>>>(X, n, lo, leaf_sums, L, rmi.leaves);
  count_launch();
  if (n) {
    const uint32_t blocks = (n + kRmiBlock - 1) / kRmiBlock;
    k_rmi_errors<<<blocks, kRmiBlock, 0, st>>>(X, n, ra, rb, L, rmi.leaves);
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
