// The database sort of bits_build_db and bits_sort_intervals_noalloc:
// B_S <- starts, B_E <- ends, each sorted (Algorithm 2's two Sort steps;
// Sec. "Parallel BITS" relies on a GPU radix sort for them).  Keys only, LSD,
// 8-bit digits.
//
//   * k_split_hist reads the interval pairs once, validates them (end >
//     start), writes the starts and the ends into two plain arrays, and
//     builds all eight digit histograms (4 digits x 2 arrays) in the same
//     pass.  The host reads the histograms once and skips every pass whose
//     digit is the same for all keys.
//   * k_sweep_keys runs one digit pass for both arrays in one persistent
//     launch (two CTAs of 512 threads per SM).  Tiles of 8192 keys are
//     handed out by an atomic ticket, alternating between the two arrays.
//     While a CTA works on one tile, the next tile it took is already on
//     its way into shared memory by a TMA bulk copy (cp.async.bulk,
//     completion on an mbarrier), so the keys of a tile are never waited for
//     in registers.  Three tile buffers rotate: the tile being ranked, the
//     tile in flight, and the staging area in which the ranked tile is laid
//     out in digit order.  Ranking is stable: the lanes with the same digit
//     come from the warp's peer table (sort_common.cuh), kept in the staging
//     slot while it is free; their lowest lane adds their number to the
//     warp's 16-bit counter of that digit (two digits per 32-bit word);
//     warps then take exclusive offsets per digit.  A tile publishes its digit counts at
//     once and gathers the prefix of earlier tiles by decoupled look-back
//     (sort_common.cuh); the staged keys then go out in runs of one digit.
//     Every wait is bounded (DEV_ERR_TIMEOUT), and a scatter index outside
//     the array is reported as DEV_ERR_INTERNAL instead of being written.
//
// Traffic per interval: 8 B read + 8 B written by the split, then per active
// pass 8 B read + 8 B written (both arrays), plus the look-back words (256
// per 8192-key tile and pass, 1/8 B per key).
#include "radix_sort.cuh"
#include "sort_common.cuh"

namespace bits {
namespace {

constexpr int kSplitBlock = 512;
constexpr int kSkBlock = 512;
constexpr int kSkWarps = kSkBlock / 32;
constexpr int kSkKpt = 16;
constexpr int kSkTile = kSkBlock * kSkKpt;  // 8192 keys
static_assert(kSkTile == (int)kRadixTileKeys, "look-back tables are sized per 8192-key tile");
constexpr int kSkBufs = 3;
constexpr int kSkCtasPerSm = 2;
constexpr int kSkCntWords = (kRadix + 2) / 2;  // digits 0..256 (256: empty lane) as 16-bit halves

// Shared-memory layout of k_sweep_keys, in 32-bit words.
constexpr int kOffCnt = kSkBufs * kSkTile;                  // [warps][kSkCntWords]
constexpr int kOffDbase = kOffCnt + kSkWarps * kSkCntWords;  // [2 arrays][256]
constexpr int kOffTstart = kOffDbase + 2 * kRadix;
constexpr int kOffGbase = kOffTstart + kRadix;
constexpr int kOffTcount = kOffGbase + kRadix;
constexpr int kOffScan = kOffTcount + kRadix;               // [8]
constexpr int kOffTix = kOffScan + 8;                       // [2] tickets (current, next)
constexpr int kOffBar = kOffTix + 2;                        // [3] mbarriers, 8 bytes each
constexpr int kSmemWords = kOffBar + 2 * kSkBufs;
static_assert(kOffBar % 2 == 0, "mbarriers need 8-byte alignment");
static_assert(kSkWarps * kPeerTableWords <= kSkTile, "peer tables fit in a tile slot");
constexpr size_t kSmemBytes = sizeof(uint32_t) * kSmemWords;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

// Arm the barrier for `bytes` of bulk-copy data (one arrival: the caller).
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

// One bulk copy global -> shared of `bytes` (16-byte aligned, multiple of 16)
// that completes on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__global__ void __launch_bounds__(kSplitBlock)
k_split_hist(const uint2* __restrict__ b, uint32_t n, uint32_t* __restrict__ out_s,
             uint32_t* __restrict__ out_e, uint32_t* __restrict__ hist,
             uint32_t* __restrict__ err) {
  __shared__ uint32_t sh[2 * kPasses * kRadix];
  for (int i = threadIdx.x; i < 2 * kPasses * kRadix; i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  bool bad = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint2 v = b[i];
    bad |= !(v.x < v.y);
    out_s[i] = v.x;
    out_e[i] = v.y;
    #pragma unroll
    for (int p = 0; p < kPasses; ++p) {
      atomicAdd(&sh[p * kRadix + ((v.x >> (8 * p)) & 255u)], 1u);
      atomicAdd(&sh[(kPasses + p) * kRadix + ((v.y >> (8 * p)) & 255u)], 1u);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_dev_error(err, DEV_ERR_INVALID);
  for (int i = threadIdx.x; i < 2 * kPasses * kRadix; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

struct SkJob {
  const uint32_t* in;    // keys before this pass
  uint32_t* out;         // keys after this pass
  const uint32_t* hist;  // [256] counts of this pass's digit over all n keys
  uint32_t* status;      // [tiles][256] look-back words, zeroed
  int shift;             // 8 * digit
  int bulk;              // `in` is 16-byte aligned: full tiles arrive by bulk copy
};
struct SkJobs {
  SkJob j[2];
  uint32_t n_jobs;       // 1 or 2
  uint32_t tiles;        // tiles per array
  uint32_t* ticket;      // zeroed
};

// Iterations of a bounded wait on a bulk copy's mbarrier (each try_wait may
// itself suspend the thread for a short, hardware-chosen time).
constexpr uint32_t kMbarSpinLimit = 1u << 20;

__global__ void __launch_bounds__(kSkBlock, kSkCtasPerSm)
k_sweep_keys(SkJobs J, uint32_t n, uint32_t* __restrict__ err) {
  extern __shared__ __align__(128) uint32_t sm[];
  uint32_t* s_cnt = sm + kOffCnt;
  uint32_t* s_dbase = sm + kOffDbase;
  uint32_t* s_tstart = sm + kOffTstart;
  uint32_t* s_gbase = sm + kOffGbase;
  uint32_t* s_tcount = sm + kOffTcount;
  uint32_t* s_scan = sm + kOffScan;
  volatile uint32_t* s_tix = sm + kOffTix;
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(sm + kOffBar);

  const unsigned tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  const uint32_t two = J.n_jobs == 2 ? 1u : 0u;
  const uint32_t total = J.tiles << two;
  // Both jobs' fields in registers; a ticket selects one of them.
  const uint32_t* const in0 = J.j[0].in;
  const uint32_t* const in1 = J.j[1].in;
  const int bulk0 = J.j[0].bulk, bulk1 = J.j[1].bulk;

  // Digit bases of this pass: exclusive prefix of each array's histogram.
  for (uint32_t jb = 0; jb <= two; ++jb) {
    const uint32_t* hist = jb ? J.j[1].hist : J.j[0].hist;
    const uint32_t h = tid < (unsigned)kRadix ? hist[tid] : 0u;
    const uint32_t x = scan256_excl(h, s_scan);
    if (tid < (unsigned)kRadix) s_dbase[jb * kRadix + tid] = x;
  }

  // Thread 0 takes tickets and starts the bulk copies; a ticket t is tile
  // t / 2 of array t % 2 (tile t of the one array when there is one).
  auto start_copy = [&](uint32_t t, int slot) {
    const uint32_t jb = t & two;
    const uint32_t tile = t >> two;
    if ((jb ? bulk1 : bulk0) && (uint64_t)(tile + 1) * kSkTile <= n) {
      // Order this CTA's earlier generic reads of the slot before the copy.
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect(&s_bar[slot], kSkTile * 4u);
      bulk_load(sm + slot * kSkTile, (jb ? in1 : in0) + (size_t)tile * kSkTile, kSkTile * 4u,
                &s_bar[slot]);
    }
  };
  if (tid == 0) {
    for (int k = 0; k < kSkBufs; ++k) mbar_init(&s_bar[k]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const uint32_t t = atomicAdd(J.ticket, 1u);
    s_tix[0] = t;
    if (t < total) start_copy(t, 0);
  }
  __syncthreads();

  uint32_t phase = 0u;  // bit k: parity of the next completion of slot k's barrier
  int L = 0;            // slot of the tile being ranked; L+1 in flight, L+2 staging
  for (uint32_t q = 0;; ++q) {
    const uint32_t cur = s_tix[q & 1u];
    if (cur >= total) break;
    const int P = L == 2 ? 0 : L + 1, S = P == 2 ? 0 : P + 1;
    if (tid == 0) {
      const uint32_t t = atomicAdd(J.ticket, 1u);
      s_tix[(q + 1) & 1u] = t;
      if (t < total) start_copy(t, P);
    }
    const uint32_t jb = cur & two;
    const uint32_t tile = cur >> two;
    const uint32_t* in = jb ? in1 : in0;
    uint32_t* out = jb ? J.j[1].out : J.j[0].out;
    uint32_t* status = jb ? J.j[1].status : J.j[0].status;
    const int shift = jb ? J.j[1].shift : J.j[0].shift;
    const int bulk = jb ? bulk1 : bulk0;
    const uint32_t base = tile * (uint32_t)kSkTile;
    const uint32_t valid = min((uint32_t)kSkTile, n - base);
    const bool full = valid == (uint32_t)kSkTile;
    uint32_t* buf_l = sm + L * kSkTile;
    uint32_t* buf_s = sm + S * kSkTile;

    if (full && bulk) {
      uint32_t spins = 0u;
      while (!mbar_try_wait(&s_bar[L], (phase >> L) & 1u)) {
        if (++spins > kMbarSpinLimit) {
          set_dev_error(err, DEV_ERR_TIMEOUT);
          break;
        }
      }
      phase ^= 1u << L;
    } else {
      for (uint32_t i = tid; i < valid; i += kSkBlock) buf_l[i] = in[base + i];
    }
    for (uint32_t i = tid; i < (uint32_t)(kSkWarps * kSkCntWords); i += kSkBlock) s_cnt[i] = 0u;
    // The staging slot holds the warps' peer tables until the tile is staged.
    for (uint32_t i = tid; i < (uint32_t)(kSkWarps * kPeerTableWords); i += kSkBlock) buf_s[i] = 0u;
    __syncthreads();

    // Stable rank of each key among the keys of its warp with the same digit
    // (positions w * 512 + k * 32 + lane, in that order); two 16-bit ranks
    // share a register.
    const uint32_t wbase = w * 32u * kSkKpt;
    uint32_t* wcnt = s_cnt + w * kSkCntWords;
    uint32_t rank2[kSkKpt / 2];
    #pragma unroll
    for (int k = 0; k < kSkKpt / 2; ++k) rank2[k] = 0u;
    #pragma unroll
    for (int h = 0; h < 2; ++h) {
      constexpr int kH = kSkKpt / 2;
      uint32_t lead[kH];
      unsigned peers_k[kH];
      #pragma unroll
      for (int kk = 0; kk < kH; ++kk) {
        const int k = h * kH + kk;
        const uint32_t pos = wbase + k * 32u + lane;
        const uint32_t d = pos < valid ? ((buf_l[pos] >> shift) & 255u) : (uint32_t)kRadix;
        const unsigned peers = peers_by_table(buf_s + w * kPeerTableWords, d);
        peers_k[kk] = peers;
        lead[kk] = 0u;
        if ((int)lane == __ffs(peers) - 1) {
          const uint32_t sh16 = (d & 1u) << 4;
          lead[kk] = (atomicAdd(wcnt + (d >> 1), (uint32_t)__popc(peers) << sh16) >> sh16) & 0xFFFFu;
        }
      }
      #pragma unroll
      for (int kk = 0; kk < kH; ++kk) {
        const int k = h * kH + kk;
        const uint32_t b0 = __shfl_sync(0xFFFFFFFFu, lead[kk], __ffs(peers_k[kk]) - 1);
        rank2[k >> 1] |= (b0 + __popc(peers_k[kk] & lanemask_lt())) << (16 * (k & 1));
      }
    }
    __syncthreads();

    // Per digit pair: exclusive offsets of the warps (packed, no carry: every
    // count is below 2^16) and the tile's count of each digit.
    if (tid < (unsigned)kSkCntWords) {
      uint32_t run = 0u;
      #pragma unroll
      for (int ww = 0; ww < kSkWarps; ++ww) {
        const uint32_t c = s_cnt[ww * kSkCntWords + tid];
        s_cnt[ww * kSkCntWords + tid] = run;
        run += c;
      }
      if (tid < (unsigned)(kRadix / 2)) {
        s_tcount[2 * tid] = run & 0xFFFFu;
        s_tcount[2 * tid + 1] = run >> 16;
      }
    }
    __syncthreads();
    const uint32_t tcount = tid < (unsigned)kRadix ? s_tcount[tid] : 0u;
    if (tid < (unsigned)kRadix) {
      // Publish this tile's counts at once so later tiles can look back.
      volatile uint32_t* st = status + (size_t)tile * kRadix + tid;
      *st = (tile == 0 ? kFlagPre : kFlagAgg) | tcount;
    }
    const uint32_t tstart = scan256_excl(tcount, s_scan);
    if (tid < (unsigned)kRadix) {
      s_tstart[tid] = tstart;
      if (tile == 0) s_gbase[tid] = s_dbase[jb * kRadix + tid] - tstart;
    }
    __syncthreads();
    // Fold the tile's digit starts into the warps' packed offsets, so that
    // staging a key reads one word (both halves stay below 2^16: every
    // position is inside the tile).
    if (tid < (unsigned)(kRadix / 2)) {
      const uint32_t add = s_tstart[2 * tid] | (s_tstart[2 * tid + 1] << 16);
      #pragma unroll
      for (int ww = 0; ww < kSkWarps; ++ww) s_cnt[ww * kSkCntWords + tid] += add;
    }
    __syncthreads();

    // Stage the tile in digit order.
    #pragma unroll
    for (int k = 0; k < kSkKpt; ++k) {
      const uint32_t pos = wbase + k * 32u + lane;
      if (pos < valid) {
        const uint32_t key = buf_l[pos];
        const uint32_t d = (key >> shift) & 255u;
        const uint32_t r = (rank2[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
        const uint32_t at = ((wcnt[d >> 1] >> ((d & 1u) << 4)) & 0xFFFFu) + r;
        if (at < (uint32_t)kSkTile) buf_s[at] = key;
      }
    }
    if (tile > 0 && tid < (unsigned)kRadix) {
      const uint32_t excl = lookback_excl(status, tile, tid, err);
      s_gbase[tid] = s_dbase[jb * kRadix + tid] + excl - tstart;
      volatile uint32_t* st = status + (size_t)tile * kRadix + tid;
      *st = kFlagPre | ((excl + tcount) & kValMask);
    }
    __syncthreads();

    bool oob = false;
    for (uint32_t i = tid; i < valid; i += kSkBlock) {
      const uint32_t v = buf_s[i];
      const uint32_t at = s_gbase[(v >> shift) & 255u] + i;
      if (at < n) out[at] = v;
      else oob = true;
    }
    if (oob) set_dev_error(err, DEV_ERR_INTERNAL);
    L = P;
    __syncthreads();  // the staging and ranked slots are free before the next copy
  }
}

}  // namespace

bits_status radix_sort_intervals(const uint2* d_b, uint32_t n, uint32_t* out_s, uint32_t* out_e,
                                 uint32_t* d_err, RadixScratch& ws, cudaStream_t st,
                                 bool read_back) {
  if (n == 0) return BITS_OK;
  const uint32_t tiles = (n + kSkTile - 1) / kSkTile;
  const size_t status_words = (size_t)tiles * kRadix;
  BITS_CUDA_TRY(cudaMemsetAsync(ws.hist, 0, sizeof(uint32_t) * 2 * kPasses * kRadix, st));
  const int split_grid =
      std::max(1, std::min<int>(sm_count() * 4, (n + kSplitBlock - 1) / kSplitBlock));
  k_split_hist<<<split_grid, kSplitBlock, 0, st>>>(d_b, n, out_s, out_e, ws.hist, d_err);
  BITS_LAUNCH_CHECK("k_split_hist");

  // Active passes per array: a pass whose digit is the same for every key
  // keeps the order and is skipped (keys all equal: no pass at all).  That
  // takes the histograms on the host; without the read-back every pass runs
  // (the result is the same) and an invalid interval only sets d_err.
  int passes[2][kPasses], np[2] = {0, 0};
  if (read_back) {
    uint32_t h_hist[2 * kPasses * kRadix];
    uint32_t h_err = 0;
    BITS_CUDA_TRY(cudaMemcpyAsync(h_hist, ws.hist, sizeof(h_hist), cudaMemcpyDeviceToHost, st));
    BITS_CUDA_TRY(cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BITS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err & DEV_ERR_INVALID) {
      set_error("a database interval has end <= start");
      return BITS_EINVAL;
    }
    for (int a = 0; a < 2; ++a)
      for (int p = 0; p < kPasses; ++p) {
        bool constant = false;
        for (int d = 0; d < kRadix; ++d)
          if (h_hist[(a * kPasses + p) * kRadix + d] == n) constant = true;
        if (!constant) passes[a][np[a]++] = p;
      }
  } else {
    for (int a = 0; a < 2; ++a)
      for (int p = 0; p < kPasses; ++p) passes[a][np[a]++] = p;
  }
  const int steps = std::max(np[0], np[1]);
  if (steps == 0) return BITS_OK;
  BITS_CUDA_TRY(cudaMemsetAsync(ws.status, 0, sizeof(uint32_t) * status_words * 2 * steps, st));
  BITS_CUDA_TRY(cudaMemsetAsync(ws.tickets, 0, sizeof(uint32_t) * steps, st));
  const int per_sm = kernel_blocks_per_sm(reinterpret_cast<const void*>(k_sweep_keys), kSkBlock,
                                          kSmemBytes, kSkCtasPerSm);
  uint32_t* outs[2] = {out_s, out_e};
  uint32_t* tmps[2] = {ws.tmp_s, ws.tmp_e};
  uint32_t* cur[2] = {out_s, out_e};  // the split left the keys in the outputs
  for (int step = 0; step < steps; ++step) {
    SkJobs J{};
    uint32_t nj = 0;
    for (int a = 0; a < 2; ++a) {
      if (step >= np[a]) continue;
      SkJob& jj = J.j[nj];
      jj.in = cur[a];
      jj.out = cur[a] == outs[a] ? tmps[a] : outs[a];
      jj.hist = ws.hist + (a * kPasses + passes[a][step]) * kRadix;
      jj.status = ws.status + status_words * (size_t)(2 * step + (int)nj);
      jj.shift = 8 * passes[a][step];
      jj.bulk = (reinterpret_cast<uintptr_t>(cur[a]) & 15u) == 0;
      cur[a] = jj.out;
      ++nj;
    }
    J.n_jobs = nj;
    J.tiles = tiles;
    J.ticket = ws.tickets + step;
    const uint32_t grid = std::min<uint32_t>(tiles * nj, (uint32_t)(per_sm * sm_count()));
    k_sweep_keys<<<grid, kSkBlock, kSmemBytes, st>>>(J, n, d_err);
    BITS_LAUNCH_CHECK("k_sweep_keys");
  }
  // An odd number of passes leaves an array in its ping-pong buffer.
  for (int a = 0; a < 2; ++a)
    if (cur[a] != outs[a])
      BITS_CUDA_TRY(cudaMemcpyAsync(outs[a], cur[a], sizeof(uint32_t) * n,
                                    cudaMemcpyDeviceToDevice, st));
  return BITS_OK;
}

}  // namespace bits
