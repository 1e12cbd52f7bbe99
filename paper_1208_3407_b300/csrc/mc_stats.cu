// Summary of Monte-Carlo tests (Sec. "Monte Carlo Simulations" tally, Sec.
// "Novel genomic relationships" / Fig. 3 score): for each test, k_ge = #{T_s
// >= observed}, k_le = #{T_s <= observed}, the two middle totals (ranks
// floor((N-1)/2) and floor(N/2) of the sorted totals), the enrichment and
// depletion p-values and the score log2(observed / median).
//
// One CTA per test.  The middles come from a most-significant-digit radix
// select over the 64-bit totals, both ranks in the same passes: a pass
// histograms one byte of the totals whose higher bytes match the prefix
// selected so far, and a warp per rank scans the 256 bins to pick the next
// byte.  Shuffled totals cluster tightly, so the select starts at the
// highest byte in which the smallest and largest total differ (every total
// shares the bytes above it): typically two or three passes over N totals
// that sit in L2.  Histogram updates are warp-aggregated (match_any), since
// clustered totals put most of a pass into a few bins.
#include "common.cuh"
#include "mc_stats.cuh"

namespace bits {
namespace {

constexpr int kStatBlock = 512;

__device__ __forceinline__ void hist_add(uint32_t* h, uint32_t bin, bool on) {
  const unsigned act = __ballot_sync(0xFFFFFFFFu, on);
  if (!on) return;
  const unsigned peers = __match_any_sync(act, bin);
  if ((peers & lanemask_lt()) == 0) atomicAdd(h + bin, (uint32_t)__popc(peers));
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}

__global__ void __launch_bounds__(kStatBlock)
k_mc_summary(const unsigned long long* __restrict__ totals, uint32_t n,
             const unsigned long long* __restrict__ observed, bits_mc_stat* __restrict__ out) {
  __shared__ uint32_t s_hist[2][256];
  __shared__ unsigned long long s_red[32];
  __shared__ unsigned long long s_mm[2][kStatBlock / 32];
  __shared__ unsigned long long s_prefix[2];
  __shared__ uint32_t s_rank[2];
  const unsigned long long* T = totals + (size_t)blockIdx.x * n;
  const unsigned long long obs = observed[blockIdx.x];
  const unsigned w = threadIdx.x >> 5, lane = lane_id();

  // Pass 0: tallies, smallest and largest total.
  unsigned long long kge = 0, kle = 0, lo = ~0ull, hi = 0;
  for (uint32_t i = threadIdx.x; i < n; i += kStatBlock) {
    const unsigned long long v = T[i];
    kge += v >= obs;
    kle += v <= obs;
    lo = min(lo, v);
    hi = max(hi, v);
  }
  lo = warp_min_u64(lo);
  hi = warp_max_u64(hi);
  if (lane == 0) {
    s_mm[0][w] = lo;
    s_mm[1][w] = hi;
  }
  kge = block_sum_u64(kge, s_red);
  __syncthreads();
  const unsigned long long kge_all = kge;  // valid in thread 0
  kle = block_sum_u64(kle, s_red);
  if (threadIdx.x == 0) {
    unsigned long long a = ~0ull, b = 0;
    for (int k = 0; k < kStatBlock / 32; ++k) {
      a = min(a, s_mm[0][k]);
      b = max(b, s_mm[1][k]);
    }
    // Every total shares the bytes above the highest byte where a and b differ.
    const int top = (n == 0 || a == b) ? -1 : (63 - __clzll(a ^ b)) / 8;  // highest differing byte
    const unsigned long long keep = top < 0 ? ~0ull : (top == 7 ? 0ull : (~0ull << (8 * (top + 1))));
    s_prefix[0] = s_prefix[1] = (n ? a : 0ull) & keep;
    s_rank[0] = n ? (n - 1) / 2 : 0u;
    s_rank[1] = n / 2;
    s_mm[0][0] = (unsigned long long)(top < 0 ? 0 : top + 1);  // passes left
  }
  __syncthreads();
  const int passes = (int)s_mm[0][0];
  for (int p = passes - 1; p >= 0; --p) {
    const int shift = 8 * p;
    const unsigned long long mask = (p == 7) ? 0ull : (~0ull << (shift + 8));
    for (uint32_t k = threadIdx.x; k < 512; k += kStatBlock) (&s_hist[0][0])[k] = 0u;
    __syncthreads();
    const unsigned long long p0 = s_prefix[0], p1 = s_prefix[1];
    const uint32_t n_round = (n + kStatBlock - 1) / kStatBlock * kStatBlock;
    for (uint32_t i = threadIdx.x; i < n_round; i += kStatBlock) {
      const bool in = i < n;
      const unsigned long long v = in ? T[i] : 0ull;
      const uint32_t bin = (uint32_t)(v >> shift) & 255u;
      hist_add(s_hist[0], bin, in && (v & mask) == p0);
      hist_add(s_hist[1], bin, in && (v & mask) == p1);
    }
    __syncthreads();
    if (w < 2) {
      // Lane l owns bins 8l .. 8l+7; find the bin holding rank s_rank[w].
      const uint32_t* h = s_hist[w];
      uint32_t c[8], sum = 0;
      #pragma unroll
      for (int k = 0; k < 8; ++k) {
        c[k] = h[8 * lane + k];
        sum += c[k];
      }
      uint32_t incl = sum;
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      const uint32_t r = s_rank[w];
      const uint32_t before = incl - sum;
      if (r >= before && r < incl) {  // exactly one lane: the candidates hold rank r
        uint32_t acc = before, b = 8 * lane + 7;
        bool found = false;
        #pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (!found) {
            if (r < acc + c[k]) {
              found = true;
              b = 8 * lane + k;
            } else {
              acc += c[k];
            }
          }
        }
        s_prefix[w] |= (unsigned long long)b << shift;
        s_rank[w] = r - acc;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bits_mc_stat st;
    const unsigned long long m0 = s_prefix[0], m1 = s_prefix[1];
    st.observed = obs;
    st.k_ge = kge_all;
    st.k_le = kle;
    st.median_lo = m0;
    st.median_hi = m1;
    st.p_enrich = (double)(kge_all + 1) / (double)((unsigned long long)n + 1);
    st.p_deplete = (double)(kle + 1) / (double)((unsigned long long)n + 1);
    const bool ovf = obs > (~0ull >> 1) || m0 > ~0ull - m1;
    st.log2_enrichment = ovf ? __longlong_as_double(0x7FF8000000000000ll)
                             : log2((double)(2ull * obs) / (double)(m0 + m1));
    out[blockIdx.x] = st;
  }
}

}  // namespace

bits_status launch_mc_summary(const uint64_t* d_totals, uint32_t n_shuffles, uint32_t n_tests,
                              const uint64_t* d_observed, bits_mc_stat* d_stats, cudaStream_t st) {
  if (n_tests == 0) return BITS_OK;
  k_mc_summary<<<n_tests, kStatBlock, 0, st>>>(
      reinterpret_cast<const unsigned long long*>(d_totals), n_shuffles,
      reinterpret_cast<const unsigned long long*>(d_observed), d_stats);
  BITS_LAUNCH_CHECK("k_mc_summary");
  return BITS_OK;
}

}  // namespace bits
