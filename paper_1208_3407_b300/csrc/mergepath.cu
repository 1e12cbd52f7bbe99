// Merge-path form of bits_count: instead of two independent searches per
// query, the queries' keys are sorted and every sorted key is co-ranked
// against the database's sorted array by merge path (Green, McColl and
// Bader, "GPU merge path", 2012):
//     first(a) = #(B_S < a.end)        key a.end     against B_S
//     last(a)  = #(B_E < a.start + 1)  key a.start+1 against B_E
// and ICount(a) = first - last (Algorithm 1).  In the merged order of a
// sorted key array Q and the sorted array X, where X[x] comes before Q[y]
// iff X[x] < Q[y], the key Q[y] sits at position x + y and its rank is x.
//
//   1. radix_sort_pairs sorts both key arrays of the queries (with their
//      indices when per-query counts are wanted; the index's top bit marks
//      an inverted query, which counts 0).
//   2. k_mp_partition finds, by binary search on each diagonal d = t * 2048,
//      how many X keys precede position d of the merge.
//   3. k_mp_merge stages one 2048-element window of X and Q in shared
//      memory, every thread merges 8 positions sequentially and emits the
//      rank of each Q key it passes: the first pass stores first(a) into
//      counts[a], the second subtracts last(a); both add to the total.
//
// Streams |A| + |B| keys per pass instead of searching; it wins when |A| is
// comparable to |B| (and most clearly for the total alone), loses when |A|
// is much smaller than |B|.  The histogram read of the sort synchronises the
// stream once per call.
#include "count.cuh"
#include "mergepath.cuh"
#include "radix_sort.cuh"

namespace bits {
namespace {

constexpr int kMpBlock = 256;
constexpr int kMpIpt = 8;
constexpr uint32_t kMpTile = kMpBlock * kMpIpt;  // 2048 merge positions per CTA

__global__ void k_mp_partition(const uint32_t* __restrict__ X, uint32_t n,
                               const uint32_t* __restrict__ Q, uint32_t m, uint32_t tiles,
                               uint32_t* __restrict__ splits) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t <= tiles;
       t += gridDim.x * blockDim.x) {
    const uint64_t d = min((uint64_t)t * kMpTile, (uint64_t)n + m);
    uint32_t lo = d > m ? (uint32_t)(d - m) : 0u;
    uint32_t hi = (uint32_t)min(d, (uint64_t)n);
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (X[mid] < Q[d - mid - 1]) lo = mid + 1;
      else hi = mid;
    }
    splits[t] = lo;
  }
}

// PASS 0: ranks are first(a); PASS 1: ranks are last(a) (a key of 0 is
// a.start = 2^32 - 1, whose last is |B|).
template <int PASS>
__global__ void __launch_bounds__(kMpBlock)
k_mp_merge(const uint32_t* __restrict__ X, uint32_t n, const uint32_t* __restrict__ Q,
           const uint32_t* __restrict__ V, uint32_t m, const uint32_t* __restrict__ splits,
           uint32_t* __restrict__ counts, unsigned long long* __restrict__ total,
           uint32_t* __restrict__ err) {
  __shared__ uint32_t sX[kMpTile];
  __shared__ uint32_t sQ[kMpTile];
  __shared__ uint32_t sV[kMpTile];
  __shared__ unsigned long long s_red[32];
  const uint32_t t = blockIdx.x;
  const uint64_t d0 = (uint64_t)t * kMpTile;
  const uint64_t d1 = min(d0 + kMpTile, (uint64_t)n + m);
  const uint32_t x0 = splits[t], x1 = splits[t + 1];
  const uint32_t y0 = (uint32_t)(d0 - x0), y1 = (uint32_t)(d1 - x1);
  // Splits of a sorted pair of arrays always satisfy these; anything else
  // means unsorted input, reported instead of read.
  if (x1 < x0 || d1 - x1 < d0 - x0 || (uint64_t)(x1 - x0) + (d1 - x1) - (d0 - x0) > kMpTile) {
    if (threadIdx.x == 0) set_dev_error(err, DEV_ERR_INTERNAL);
    return;
  }
  const uint32_t nx = x1 - x0, ny = y1 - y0;
  for (uint32_t i = threadIdx.x; i < nx; i += blockDim.x) sX[i] = X[x0 + i];
  for (uint32_t i = threadIdx.x; i < ny; i += blockDim.x) {
    sQ[i] = Q[y0 + i];
    if (V) sV[i] = V[y0 + i];
  }
  __syncthreads();
  const uint32_t len = nx + ny;
  const uint32_t ld = min((uint32_t)threadIdx.x * kMpIpt, len);
  uint32_t lo = ld > ny ? ld - ny : 0u, hi = min(ld, nx);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (sX[mid] < sQ[ld - mid - 1]) lo = mid + 1;
    else hi = mid;
  }
  uint32_t x = lo, y = ld - lo;
  unsigned long long acc = 0ull;
  bool bad = false;
  for (int k = 0; k < kMpIpt && x + y < len; ++k) {
    if (x < nx && (y >= ny || sX[x] < sQ[y])) {
      ++x;
      continue;
    }
    uint32_t r = x0 + x;
    if (PASS == 1 && sQ[y] == 0u) r = n;
    bool flagged = false;
    if (V) {
      const uint32_t v = sV[y];
      const uint32_t idx = v & 0x7FFFFFFFu;
      flagged = (v >> 31) != 0u;
      if (counts) {
        if (PASS == 0) {
          counts[idx] = r;
        } else {
          counts[idx] = flagged ? 0u : counts[idx] - r;
        }
      }
    }
    if (flagged) bad = true;
    else acc += r;
    ++y;
  }
  if (PASS == 1 && __syncthreads_or(bad) && threadIdx.x == 0) set_dev_error(err, DEV_ERR_INVALID);
  const unsigned long long sum = block_sum_u64(acc, s_red);
  if (threadIdx.x == 0 && sum) atomicAdd(total, PASS == 0 ? sum : (0ull - sum));
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

bits_status launch_count_mergepath(const bits_db* db, const uint32_t* d_a, uint32_t n,
                                   uint32_t* d_counts, uint64_t* d_total, cudaStream_t st) {
  BITS_CUDA_TRY(cudaMemsetAsync(d_total, 0, sizeof(uint64_t), st));
  if (n == 0) return BITS_OK;
  if (n >= (1u << 31)) {
    set_error("bits_count (merge path): at most 2^31 - 1 queries per call");
    return BITS_EOVERFLOW;
  }
  const uint32_t nb = db->n;
  const uint32_t tiles = (uint32_t)(((uint64_t)n + nb + kMpTile - 1) / kMpTile);
  const size_t words_n = align256(sizeof(uint32_t) * n);
  const size_t sw = radix_status_words(n);
  const size_t bytes = 8 * words_n + align256(sizeof(uint32_t) * kRadixHistWords) +
                       align256(sizeof(uint32_t) * sw * 8) + 256 +
                       2 * align256(sizeof(uint32_t) * (tiles + 1));
  void* scratch = nullptr;
  {
    const bits_status as = pool_alloc(&scratch, bytes, st);
    if (as != BITS_OK) return as;
  }
  char* p = static_cast<char*>(scratch);
  auto take = [&](size_t b) {
    char* q = p;
    p += b;
    return reinterpret_cast<uint32_t*>(q);
  };
  uint32_t* keys_e = take(words_n);
  uint32_t* vals_e = take(words_n);
  uint32_t* keys_s = take(words_n);
  uint32_t* vals_s = take(words_n);
  RadixScratch ws{};
  SortSpec spec[2]{};
  spec[0].comp = 1;  // a.end, ranked in B_S
  spec[0].out_keys = keys_e;
  spec[0].tmp_keys = take(words_n);
  spec[1].comp = 0;  // a.start + 1, ranked in B_E
  spec[1].add = 1;
  spec[1].out_keys = keys_s;
  spec[1].tmp_keys = take(words_n);
  uint32_t* tmp_v0 = take(words_n);
  uint32_t* tmp_v1 = take(words_n);
  ws.hist = take(align256(sizeof(uint32_t) * kRadixHistWords));
  ws.status = take(align256(sizeof(uint32_t) * sw * 8));
  ws.tickets = take(256);
  uint32_t* splits_e = take(align256(sizeof(uint32_t) * (tiles + 1)));
  uint32_t* splits_s = take(align256(sizeof(uint32_t) * (tiles + 1)));
  ws.tmp_s = spec[0].tmp_keys;
  ws.tmp_e = spec[1].tmp_keys;
  auto done = [&](bits_status s) {
    pool_free(scratch, st);
    return s;
  };

  bool kv = d_counts != nullptr;
  for (int attempt = 0; attempt < 2; ++attempt) {
    spec[0].out_vals = kv ? vals_e : nullptr;
    spec[0].tmp_vals = kv ? tmp_v0 : nullptr;
    spec[0].flag_inverted = 1;
    spec[1].out_vals = kv ? vals_s : nullptr;
    spec[1].tmp_vals = kv ? tmp_v1 : nullptr;
    spec[1].flag_inverted = 1;
    bool inverted = false;
    bits_status s = radix_sort_pairs(reinterpret_cast<const uint2*>(d_a), n, spec, 1, db->err,
                                     ws, st, &inverted);
    if (s != BITS_OK) return done(s);
    if (kv || !inverted) break;
    kv = true;  // inverted queries must be left out of the total: redo with indices
  }

  const int pgrid = (int)std::min<uint32_t>((tiles + 1 + 255) / 256, 4096);
  k_mp_partition<<<pgrid, 256, 0, st>>>(db->bs, nb, keys_e, n, tiles, splits_e);
  count_launch();
  k_mp_partition<<<pgrid, 256, 0, st>>>(db->be, nb, keys_s, n, tiles, splits_s);
  count_launch();
  auto* tot = reinterpret_cast<unsigned long long*>(d_total);
  k_mp_merge<0><<<tiles, kMpBlock, 0, st>>>(db->bs, nb, keys_e, kv ? vals_e : nullptr, n,
                                            splits_e, d_counts, tot, db->err);
  count_launch();
  k_mp_merge<1><<<tiles, kMpBlock, 0, st>>>(db->be, nb, keys_s, kv ? vals_s : nullptr, n,
                                            splits_s, d_counts, tot, db->err);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return done(cuda_status(e, "merge-path kernels"));
  return done(BITS_OK);
}

}  // namespace bits
