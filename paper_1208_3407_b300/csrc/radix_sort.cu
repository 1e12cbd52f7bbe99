// LSD radix sort of key/value pairs drawn from interval pairs: the
// enumeration database's start order with interval indices and the merge
// path's query sort (Algorithm 2's Sort steps with values; the keys-only
// database sort of Sec. "Parallel BITS" is sort_keys.cu).
//
// Design (one GPU, HBM-bound):
//   * k_radix_hist reads the interval array once, validates it, and builds
//     all four 8-bit digit histograms of the two keys it derives from every
//     interval (each the start or the end word, plus a constant, exactly as
//     the first pass derives them).
//   * k_onesweep runs one digit pass for both key arrays in one launch.  A
//     tile of 8192 keys is ranked stably inside the CTA (per-warp peer
//     tables and digit counters in shared memory), its per-digit counts are
//     published to a decoupled look-back table, and the CTA gathers the
//     exclusive prefix of earlier tiles from that table (sort_common.cuh).
//     Keys and values are staged in digit order in shared memory so that
//     stores of one digit are contiguous.  The first pass reads its key
//     straight out of the interval array; its value is the interval's index
//     (top bit set if the interval is inverted).  Tiles take ticket numbers
//     in launch order, so a tile only waits on tiles that already run; every
//     wait is bounded and reports DEV_ERR_TIMEOUT.
//   * Passes whose digit is the same for every key are skipped (the host
//     reads the histograms once, together with the validation flag).
//
// Traffic per key: 8 B pair read for the histogram (shared by both arrays),
// 8 B pair read in the first pass, then passes x (4 B read + 4 B write),
// doubled for values.
#include "common.cuh"
#include "radix_sort.cuh"
#include "sort_common.cuh"

namespace bits {
namespace {

constexpr int kHistBlock = 512;
constexpr int kSwBlock = 512;
constexpr int kSwWarps = kSwBlock / 32;
constexpr int kSwKpt = 16;
constexpr int kSwTile = kSwBlock * kSwKpt;  // 8192 keys
static_assert(kSwTile == (int)kRadixTileKeys, "tile size shared with the look-back sizing");
static_assert(kSwWarps * kPeerTableWords <= kSwTile, "peer tables fit in the staging area");
constexpr int kCnt = kRadix + 1;  // per-warp counters: 256 digits + the tail's empty lanes

// validate: 0 = database (end > start required, else DEV_ERR_INVALID),
//           1 = queries (end < start sets *inv, not an error here).
__global__ void __launch_bounds__(kHistBlock)
k_radix_hist(const uint2* __restrict__ b, uint32_t n, int comp0, uint32_t add0, int comp1,
             uint32_t add1, int validate, uint32_t* __restrict__ hist, uint32_t* __restrict__ err,
             uint32_t* __restrict__ inv) {
  __shared__ uint32_t sh[2 * kPasses * kRadix];
  for (int i = threadIdx.x; i < 2 * kPasses * kRadix; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  bool bad = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint2 v = b[i];
    bad |= validate ? (v.y < v.x) : !(v.x < v.y);
    const uint32_t k0 = (comp0 ? v.y : v.x) + add0, k1 = (comp1 ? v.y : v.x) + add1;
    #pragma unroll
    for (int p = 0; p < kPasses; ++p) {
      atomicAdd(&sh[p * kRadix + ((k0 >> (8 * p)) & 255u)], 1u);
      atomicAdd(&sh[(kPasses + p) * kRadix + ((k1 >> (8 * p)) & 255u)], 1u);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) {
    if (validate) atomicOr(inv, 1u);
    else set_dev_error(err, DEV_ERR_INVALID);
  }
  for (int i = threadIdx.x; i < 2 * kPasses * kRadix; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

struct SweepJob {
  const uint32_t* in_keys;  // keys of the previous pass, or NULL on the first pass
  const uint32_t* in_vals;  // values of the previous pass (key/value mode)
  const uint2* aos;         // interval pairs (first pass)
  uint32_t* out_keys;
  uint32_t* out_vals;
  const uint32_t* hist;     // [256] digit histogram of this pass
  uint32_t* status;         // [tiles][256] look-back words, zeroed
  uint32_t* ticket;         // zeroed
  int comp;                 // first pass: 0 = start word, 1 = end word
  uint32_t add;             // first pass: constant added to the word
  int flag_inv;             // first pass: mark inverted intervals in the value
  int shift;
};
struct SweepJobs {
  SweepJob j[2];
};

template <bool KV>
__global__ void __launch_bounds__(kSwBlock, 2)
k_onesweep(SweepJobs jobs, uint32_t n, uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* s_stage = sm;
  uint32_t* s_vstage = sm + kSwTile;  // key/value mode only
  uint32_t* s_wcnt = sm + (KV ? 2 : 1) * kSwTile;  // [warps][kCnt]: per-warp digit counters
  uint32_t* s_gbase = s_wcnt + kSwWarps * kCnt;
  uint32_t* s_w = s_gbase + kRadix;
  uint32_t* s_tile = s_w + kRadix / 32;

  const bool y1 = blockIdx.y != 0;
  const SweepJob& J0 = jobs.j[0];
  const SweepJob& J1 = jobs.j[1];
  const uint32_t* in_keys = y1 ? J1.in_keys : J0.in_keys;
  const uint32_t* in_vals = y1 ? J1.in_vals : J0.in_vals;
  const uint2* aos = y1 ? J1.aos : J0.aos;
  uint32_t* out_keys = y1 ? J1.out_keys : J0.out_keys;
  uint32_t* out_vals = y1 ? J1.out_vals : J0.out_vals;
  const uint32_t* hist = y1 ? J1.hist : J0.hist;
  uint32_t* status = y1 ? J1.status : J0.status;
  uint32_t* ticket = y1 ? J1.ticket : J0.ticket;
  const int comp = y1 ? J1.comp : J0.comp;
  const uint32_t add = y1 ? J1.add : J0.add;
  const int flag_inv = y1 ? J1.flag_inv : J0.flag_inv;
  const int shift = y1 ? J1.shift : J0.shift;

  const unsigned tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  if (tid == 0) *s_tile = atomicAdd(ticket, 1u);
  for (int i = tid; i < kSwWarps * kCnt; i += kSwBlock) s_wcnt[i] = 0u;
  for (int i = tid; i < kSwWarps * kPeerTableWords; i += kSwBlock) s_stage[i] = 0u;
  const uint32_t hcount = tid < kRadix ? hist[tid] : 0u;
  const uint32_t dbase = scan256_excl(hcount, s_w);  // also publishes *s_tile / s_wcnt
  const uint32_t tile = *s_tile;
  const uint32_t tile_base = tile * (uint32_t)kSwTile;
  const uint32_t warp_base = tile_base + w * 32u * kSwKpt;

  uint32_t key[kSwKpt];
  #pragma unroll
  for (int k = 0; k < kSwKpt; ++k) {
    const uint32_t idx = warp_base + k * 32u + lane;
    uint32_t v = 0u;
    if (idx < n) {
      if (in_keys) {
        v = in_keys[idx];
      } else {
        const uint2 p = aos[idx];
        v = (comp ? p.y : p.x) + add;
      }
    }
    key[k] = v;
  }

  // Stable rank of every key among the keys of its warp with the same digit
  // (< 32 * kSwKpt, so two 16-bit ranks share a register).  The lanes that
  // share a digit come from the warp's peer table (sort_common.cuh; the
  // tail's empty lanes use digit 256), kept in the staging area until the
  // tile is staged; the lowest of them adds their number to the warp's
  // counter with one shared-memory atomic and passes the old value on.  The atomics of one warp are performed in program
  // order, so ranks follow key order within the warp.
  uint32_t rank2[kSwKpt / 2];
  #pragma unroll
  for (int k = 0; k < kSwKpt / 2; ++k) rank2[k] = 0u;
  #pragma unroll
  for (int h = 0; h < 2; ++h) {
    constexpr int kH = kSwKpt / 2;
    uint32_t lead_base[kH];
    unsigned peers_k[kH];
    #pragma unroll
    for (int kk = 0; kk < kH; ++kk) {
      const int k = h * kH + kk;
      const uint32_t idx = warp_base + k * 32u + lane;
      const uint32_t d = idx < n ? ((key[k] >> shift) & 255u) : 256u;
      const unsigned peers = peers_by_table(s_stage + w * kPeerTableWords, d);
      peers_k[kk] = peers;
      lead_base[kk] = 0u;
      if ((int)lane == __ffs(peers) - 1)
        lead_base[kk] = atomicAdd(s_wcnt + w * kCnt + d, (unsigned)__popc(peers));
    }
    #pragma unroll
    for (int kk = 0; kk < kH; ++kk) {
      const int k = h * kH + kk;
      const uint32_t base = __shfl_sync(0xFFFFFFFFu, lead_base[kk], __ffs(peers_k[kk]) - 1);
      rank2[k / 2] |= (base + __popc(peers_k[kk] & lanemask_lt())) << (16 * (k & 1));
    }
  }
  __syncthreads();

  // Per digit: exclusive offsets of each warp, and the tile's count.
  uint32_t tcount = 0u;
  if (tid < kRadix) {
    #pragma unroll
    for (int ww = 0; ww < kSwWarps; ++ww) {
      const uint32_t c = s_wcnt[ww * kCnt + tid];
      s_wcnt[ww * kCnt + tid] = tcount;
      tcount += c;
    }
    // Publish this tile's count as early as possible.
    volatile uint32_t* st = status + (size_t)tile * kRadix + tid;
    *st = (tile == 0 ? kFlagPre : kFlagAgg) | tcount;
  }
  const uint32_t tstart = scan256_excl(tcount, s_w);
  if (tid < kRadix) {
    // Each warp's offset of this digit becomes its position in the tile,
    // so that staging a key reads one word.
    #pragma unroll
    for (int ww = 0; ww < kSwWarps; ++ww) s_wcnt[ww * kCnt + tid] += tstart;
    if (tile == 0) s_gbase[tid] = dbase - tstart;
  }
  __syncthreads();

  // Stage the tile's keys (and values) in digit order.
  #pragma unroll
  for (int k = 0; k < kSwKpt; ++k) {
    const uint32_t idx = warp_base + k * 32u + lane;
    if (idx < n) {
      const uint32_t d = (key[k] >> shift) & 255u;
      const uint32_t r = (rank2[k / 2] >> (16 * (k & 1))) & 0xFFFFu;
      const uint32_t at = s_wcnt[w * kCnt + d] + r;
      if (at < (uint32_t)kSwTile) {
        s_stage[at] = key[k];
        if (KV) {
          uint32_t v;
          if (in_keys) {
            v = in_vals[idx];
          } else {
            v = idx;
            if (flag_inv) {
              const uint2 p = aos[idx];
              if (p.y < p.x) v |= 0x80000000u;
            }
          }
          s_vstage[at] = v;
        }
      }
    }
  }

  // Decoupled look-back (sort_common.cuh), one thread per digit.
  if (tile > 0 && tid < kRadix) {
    const uint32_t excl = lookback_excl(status, tile, tid, err);
    s_gbase[tid] = dbase + excl - tstart;
    volatile uint32_t* st = status + (size_t)tile * kRadix + tid;
    *st = kFlagPre | ((excl + tcount) & kValMask);
  }
  __syncthreads();

  const uint32_t valid_here = min((uint32_t)kSwTile, n - tile_base);
  bool oob = false;
  for (uint32_t i = tid; i < valid_here; i += kSwBlock) {
    const uint32_t v = s_stage[i];
    const uint32_t at = s_gbase[(v >> shift) & 255u] + i;
    if (at < n) {
      out_keys[at] = v;
      if (KV) out_vals[at] = s_vstage[i];
    } else {
      oob = true;
    }
  }
  if (oob) set_dev_error(err, DEV_ERR_INTERNAL);
}

size_t sweep_smem(bool kv) {
  return sizeof(uint32_t) *
         ((kv ? 2 : 1) * kSwTile + kSwWarps * kCnt + kRadix + kRadix / 32 + 4);
}

// Raises k_onesweep's dynamic shared-memory limit on the current device
// (once per device, through the per-device cache).
template <bool KV>
void prepare_sweep() {
  kernel_blocks_per_sm(reinterpret_cast<const void*>(k_onesweep<KV>), kSwBlock, sweep_smem(KV));
}

}  // namespace

size_t radix_status_words(uint32_t n) { return radix_status_words_max(n); }

bits_status radix_sort_pairs(const uint2* d_src, uint32_t n, const SortSpec spec[2], int validate,
                             uint32_t* d_err, RadixScratch& ws, cudaStream_t st,
                             bool* any_inverted) {
  if (any_inverted) *any_inverted = false;
  if (n == 0) return BITS_OK;
  const bool kv = spec[0].out_vals != nullptr;
  const uint32_t tiles = (n + kSwTile - 1) / kSwTile;
  const size_t status_words = (size_t)tiles * kRadix;

  BITS_CUDA_TRY(cudaMemsetAsync(ws.hist, 0, sizeof(uint32_t) * (2 * kPasses * kRadix + 1), st));
  uint32_t* d_inv = ws.hist + 2 * kPasses * kRadix;
  const int hist_grid = std::max(1, std::min<int>(sm_count() * 4, (n + kHistBlock - 1) / kHistBlock));
  k_radix_hist<<<hist_grid, kHistBlock, 0, st>>>(d_src, n, spec[0].comp, spec[0].add,
                                                 spec[1].comp, spec[1].add, validate, ws.hist,
                                                 d_err, d_inv);
  BITS_LAUNCH_CHECK("k_radix_hist");

  uint32_t h_hist[2 * kPasses * kRadix + 1];
  uint32_t h_err = 0;
  BITS_CUDA_TRY(cudaMemcpyAsync(h_hist, ws.hist, sizeof(h_hist), cudaMemcpyDeviceToHost, st));
  BITS_CUDA_TRY(cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  BITS_CUDA_TRY(cudaStreamSynchronize(st));
  if (!validate && (h_err & DEV_ERR_INVALID)) {
    set_error("a database interval has end <= start");
    return BITS_EINVAL;
  }
  if (any_inverted) *any_inverted = h_hist[2 * kPasses * kRadix] != 0;

  // Active passes per array: a pass whose digit is constant keeps the order.
  // Every array keeps at least one pass, which moves it out of the pairs.
  int passes[2][kPasses], np[2] = {0, 0};
  for (int a = 0; a < 2; ++a) {
    for (int p = 0; p < kPasses; ++p) {
      bool constant = false;
      for (int d = 0; d < kRadix; ++d)
        if (h_hist[(a * kPasses + p) * kRadix + d] == n) constant = true;
      if (!constant) passes[a][np[a]++] = p;
    }
    if (np[a] == 0) passes[a][np[a]++] = 0;
  }
  const int steps = std::max(np[0], np[1]);
  BITS_CUDA_TRY(cudaMemsetAsync(ws.status, 0, sizeof(uint32_t) * status_words * 2 * steps, st));
  BITS_CUDA_TRY(cudaMemsetAsync(ws.tickets, 0, sizeof(uint32_t) * 2 * kPasses, st));
  if (kv) prepare_sweep<true>();
  else prepare_sweep<false>();

  const uint32_t* cur_k[2] = {nullptr, nullptr};
  const uint32_t* cur_v[2] = {nullptr, nullptr};
  for (int step = 0; step < steps; ++step) {
    SweepJobs jobs{};
    int nj = 0;
    for (int a = 0; a < 2; ++a) {
      if (step >= np[a]) continue;
      // Ping-pong so that the array's last active pass lands in the output.
      const bool to_out = (np[a] - 1 - step) % 2 == 0;
      SweepJob& J = jobs.j[nj];
      J.in_keys = cur_k[a];
      J.in_vals = cur_v[a];
      J.aos = d_src;
      J.out_keys = to_out ? spec[a].out_keys : spec[a].tmp_keys;
      J.out_vals = to_out ? spec[a].out_vals : spec[a].tmp_vals;
      J.hist = ws.hist + (a * kPasses + passes[a][step]) * kRadix;
      J.status = ws.status + status_words * (size_t)(2 * step + a);
      J.ticket = ws.tickets + 2 * step + a;
      J.comp = spec[a].comp;
      J.add = spec[a].add;
      J.flag_inv = spec[a].flag_inverted;
      J.shift = 8 * passes[a][step];
      cur_k[a] = J.out_keys;
      cur_v[a] = J.out_vals;
      ++nj;
    }
    dim3 grid(tiles, nj);
    if (kv) k_onesweep<true><<<grid, kSwBlock, sweep_smem(true), st>>>(jobs, n, d_err);
    else k_onesweep<false><<<grid, kSwBlock, sweep_smem(false), st>>>(jobs, n, d_err);
    BITS_LAUNCH_CHECK("k_onesweep");
  }
  return BITS_OK;
}

}  // namespace bits
