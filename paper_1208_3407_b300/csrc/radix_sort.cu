// LSD radix sort of the interval starts and ends (Algorithm 2's two Sort
// steps; Sec. 2.4 relies on a GPU radix sort for them).
//
// Design (one GPU, HBM-bound):
//   * k_radix_hist reads the array-of-structures input once, validates
//     start < end, and builds all four 8-bit digit histograms of both the
//     start and the end keys (8 x 256 counters).
//   * k_onesweep runs one digit pass for both arrays in one launch.  A tile
//     of 8192 keys is ranked stably inside the CTA (warp match-any per key),
//     its per-digit counts are published to a decoupled look-back table, the
//     CTA gathers the exclusive prefix of earlier tiles from that table and
//     scatters its keys, staged in digit order in shared memory so that
//     stores of one digit are contiguous.  The first pass reads the start or
//     end word straight out of the interval array, so there is no separate
//     split step.  Tiles take ticket numbers in launch order, so a tile waits
//     only on tiles that already run; every wait is bounded and reports
//     DEV_ERR_TIMEOUT instead of hanging.
//   * Passes whose digit is the same for every key are skipped (the host
//     reads the histograms once, together with the validation flag).
//
// Traffic per key: 8 B (histogram read of the pair, shared by both arrays)
// + passes x (4 B read + 4 B write), plus 8 B/key of first-pass pair reads.
#include "common.cuh"
#include "radix_sort.cuh"

namespace bits {
namespace {

constexpr int kRadix = 256;
constexpr int kPasses = 4;
constexpr int kHistBlock = 512;
constexpr int kSwBlock = 512;
constexpr int kSwWarps = kSwBlock / 32;
constexpr int kSwKpt = 16;
constexpr int kSwTile = kSwBlock * kSwKpt;  // 8192 keys
constexpr uint32_t kFlagAgg = 1u << 30, kFlagPre = 2u << 30, kValMask = (1u << 30) - 1;

__global__ void __launch_bounds__(kHistBlock)
k_radix_hist(const uint2* __restrict__ b, uint32_t n, uint32_t* __restrict__ hist,
             uint32_t* __restrict__ err) {
  __shared__ uint32_t sh[2 * kPasses * kRadix];
  for (int i = threadIdx.x; i < 2 * kPasses * kRadix; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  bool bad = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint2 v = b[i];
    bad |= !(v.x < v.y);
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

struct SweepJob {
  const uint32_t* in;  // keys of the previous pass, or NULL on the first pass
  const uint2* aos;    // interval pairs (first pass)
  uint32_t* out;
  const uint32_t* hist;  // [256] digit histogram of this pass
  uint32_t* status;      // [tiles][256] look-back words, zeroed
  uint32_t* ticket;      // zeroed
  int comp;              // 0: start word, 1: end word
  int shift;
};
struct SweepJobs {
  SweepJob j[2];
};

// Exclusive scan of one value per thread over threads [0, 256); every
// thread of the block must call it.
__device__ __forceinline__ uint32_t scan256_excl(uint32_t v, uint32_t* s_w) {
  const unsigned lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t x = threadIdx.x < kRadix ? v : 0u;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (threadIdx.x < kRadix && lane == 31) s_w[w] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t t = lane < kRadix / 32 ? s_w[lane] : 0u;
    #pragma unroll
    for (int o = 1; o < kRadix / 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= (unsigned)o) t += y;
    }
    if (lane < kRadix / 32) s_w[lane] = t;
  }
  __syncthreads();
  const uint32_t r = (threadIdx.x < kRadix) ? (x - v + (w > 0 ? s_w[w - 1] : 0u)) : 0u;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kSwBlock, 2)
k_onesweep(SweepJobs jobs, uint32_t n, uint32_t* __restrict__ err) {
  __shared__ uint32_t s_stage[kSwTile];
  __shared__ uint16_t s_wcnt[kSwWarps][kRadix];
  __shared__ uint32_t s_tstart[kRadix];
  __shared__ uint32_t s_gbase[kRadix];
  __shared__ uint32_t s_w[kRadix / 32];
  __shared__ uint32_t s_tile;

  const bool y1 = blockIdx.y != 0;
  const uint32_t* in = y1 ? jobs.j[1].in : jobs.j[0].in;
  const uint2* aos = y1 ? jobs.j[1].aos : jobs.j[0].aos;
  uint32_t* out = y1 ? jobs.j[1].out : jobs.j[0].out;
  const uint32_t* hist = y1 ? jobs.j[1].hist : jobs.j[0].hist;
  uint32_t* status = y1 ? jobs.j[1].status : jobs.j[0].status;
  uint32_t* ticket = y1 ? jobs.j[1].ticket : jobs.j[0].ticket;
  const int comp = y1 ? jobs.j[1].comp : jobs.j[0].comp;
  const int shift = y1 ? jobs.j[1].shift : jobs.j[0].shift;

  const unsigned tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(ticket, 1u);
  {
    uint32_t* z = reinterpret_cast<uint32_t*>(&s_wcnt[0][0]);
    for (int i = tid; i < kSwWarps * kRadix / 2; i += kSwBlock) z[i] = 0u;
  }
  const uint32_t hcount = tid < kRadix ? hist[tid] : 0u;
  const uint32_t dbase = scan256_excl(hcount, s_w);  // also syncs s_tile / s_wcnt
  const uint32_t tile = s_tile;
  const uint32_t tile_base = tile * (uint32_t)kSwTile;
  const uint32_t warp_base = tile_base + w * 32u * kSwKpt;

  uint32_t key[kSwKpt];
  #pragma unroll
  for (int k = 0; k < kSwKpt; ++k) {
    const uint32_t idx = warp_base + k * 32u + lane;
    uint32_t v = 0u;
    if (idx < n) {
      if (in) {
        v = in[idx];
      } else {
        const uint2 p = aos[idx];
        v = comp ? p.y : p.x;
      }
    }
    key[k] = v;
  }

  // Stable rank of every key among the keys of its warp with the same digit
  // (< 32 * kSwKpt, so two 16-bit ranks share a register).
  uint32_t rank2[kSwKpt / 2];
  #pragma unroll
  for (int k = 0; k < kSwKpt / 2; ++k) rank2[k] = 0u;
  #pragma unroll
  for (int k = 0; k < kSwKpt; ++k) {
    const uint32_t idx = warp_base + k * 32u + lane;
    const bool valid = idx < n;
    const unsigned vmask = __ballot_sync(0xFFFFFFFFu, valid);
    const uint32_t d = (key[k] >> shift) & 255u;
    if (valid) {
      const unsigned peers = __match_any_sync(vmask, d);
      const int leader = __ffs(peers) - 1;
      uint32_t base = 0u;
      if ((int)lane == leader) {
        base = s_wcnt[w][d];
        s_wcnt[w][d] = (uint16_t)(base + __popc(peers));
      }
      base = __shfl_sync(vmask, base, leader);
      __syncwarp(vmask);
      rank2[k / 2] |= (base + __popc(peers & lanemask_lt())) << (16 * (k & 1));
    }
  }
  __syncthreads();

  // Per digit: exclusive offsets of each warp, and the tile's count.
  uint32_t tcount = 0u;
  if (tid < kRadix) {
    #pragma unroll
    for (int ww = 0; ww < kSwWarps; ++ww) {
      const uint32_t c = s_wcnt[ww][tid];
      s_wcnt[ww][tid] = (uint16_t)tcount;
      tcount += c;
    }
    // Publish this tile's count as early as possible.
    volatile uint32_t* st = status + (size_t)tile * kRadix + tid;
    *st = (tile == 0 ? kFlagPre : kFlagAgg) | tcount;
  }
  const uint32_t tstart = scan256_excl(tcount, s_w);
  if (tid < kRadix) s_tstart[tid] = tstart;
  __syncthreads();

  // Stage the tile's keys in digit order.
  #pragma unroll
  for (int k = 0; k < kSwKpt; ++k) {
    const uint32_t idx = warp_base + k * 32u + lane;
    if (idx < n) {
      const uint32_t d = (key[k] >> shift) & 255u;
      const uint32_t r = (rank2[k / 2] >> (16 * (k & 1))) & 0xFFFFu;
      const uint32_t at = s_tstart[d] + s_wcnt[w][d] + r;
      if (at < (uint32_t)kSwTile) s_stage[at] = key[k];
    }
  }

  // Decoupled look-back: exclusive prefix of this digit over earlier tiles.
  if (tid < kRadix) {
    uint32_t excl = 0u;
    if (tile > 0) {
      uint32_t t = tile - 1, spins = 0;
      while (true) {
        const uint32_t v = *(volatile const uint32_t*)(status + (size_t)t * kRadix + tid);
        const uint32_t flag = v & ~kValMask;
        if (flag == 0u) {
          if (++spins > kSpinLimit) {
            set_dev_error(err, DEV_ERR_TIMEOUT);
            break;
          }
          __nanosleep(100);
          continue;
        }
        excl += v & kValMask;
        if (flag == kFlagPre || t == 0) break;
        --t;
      }
      volatile uint32_t* st = status + (size_t)tile * kRadix + tid;
      *st = kFlagPre | ((excl + tcount) & kValMask);
    }
    s_gbase[tid] = dbase + excl - tstart;
  }
  __syncthreads();

  const uint32_t valid_here = min((uint32_t)kSwTile, n - tile_base);
  bool oob = false;
  for (uint32_t i = tid; i < valid_here; i += kSwBlock) {
    const uint32_t v = s_stage[i];
    const uint32_t at = s_gbase[(v >> shift) & 255u] + i;
    if (at < n) out[at] = v;
    else oob = true;
  }
  if (oob) set_dev_error(err, DEV_ERR_TIMEOUT);
}

}  // namespace

size_t radix_status_words(uint32_t n) {
  const uint32_t tiles = (n + kSwTile - 1) / kSwTile;
  return (size_t)tiles * kRadix;
}

bits_status radix_sort_intervals(const uint2* d_b, uint32_t n, uint32_t* out_s, uint32_t* out_e,
                                 uint32_t* d_err, RadixScratch& ws, cudaStream_t st) {
  if (n == 0) return BITS_OK;
  const uint32_t tiles = (n + kSwTile - 1) / kSwTile;
  const size_t status_words = (size_t)tiles * kRadix;

  BITS_CUDA_TRY(cudaMemsetAsync(ws.hist, 0, sizeof(uint32_t) * 2 * kPasses * kRadix, st));
  const int hist_grid = std::max(1, std::min<int>(sm_count() * 4, (n + kHistBlock - 1) / kHistBlock));
  k_radix_hist<<<hist_grid, kHistBlock, 0, st>>>(d_b, n, ws.hist, d_err);
  BITS_LAUNCH_CHECK("k_radix_hist");

  uint32_t h_hist[2 * kPasses * kRadix];
  uint32_t h_err = 0;
  BITS_CUDA_TRY(cudaMemcpyAsync(h_hist, ws.hist, sizeof(h_hist), cudaMemcpyDeviceToHost, st));
  BITS_CUDA_TRY(cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  BITS_CUDA_TRY(cudaStreamSynchronize(st));
  if (h_err & DEV_ERR_INVALID) {
    set_error("bits_build_db: a database interval has end <= start");
    return BITS_EINVAL;
  }

  // Active passes per array: a pass whose digit is constant keeps the order.
  int passes[2][kPasses], np[2] = {0, 0};
  for (int a = 0; a < 2; ++a) {
    for (int p = 0; p < kPasses; ++p) {
      bool constant = false;
      for (int d = 0; d < kRadix; ++d)
        if (h_hist[(a * kPasses + p) * kRadix + d] == n) constant = true;
      if (!constant) passes[a][np[a]++] = p;
    }
    if (np[a] == 0) passes[a][np[a]++] = 0;  // still split the keys out of the pairs
  }
  const int steps = std::max(np[0], np[1]);
  BITS_CUDA_TRY(cudaMemsetAsync(ws.status, 0, sizeof(uint32_t) * status_words * 2 * steps, st));
  BITS_CUDA_TRY(cudaMemsetAsync(ws.tickets, 0, sizeof(uint32_t) * 2 * kPasses, st));

  uint32_t* final_out[2] = {out_s, out_e};
  uint32_t* tmp[2] = {ws.tmp_s, ws.tmp_e};
  const uint32_t* cur[2] = {nullptr, nullptr};
  for (int step = 0; step < steps; ++step) {
    SweepJobs jobs{};
    int nj = 0;
    int job_array[2] = {-1, -1};
    for (int a = 0; a < 2; ++a) {
      if (step >= np[a]) continue;
      // Ping-pong so that the array's last active pass lands in final_out.
      const int remaining = np[a] - 1 - step;
      uint32_t* dst = (remaining % 2 == 0) ? final_out[a] : tmp[a];
      SweepJob& J = jobs.j[nj];
      J.in = cur[a];
      J.aos = d_b;
      J.comp = a;
      J.out = dst;
      J.hist = ws.hist + (a * kPasses + passes[a][step]) * kRadix;
      J.status = ws.status + status_words * (size_t)(2 * step + a);
      J.ticket = ws.tickets + 2 * step + a;
      J.shift = 8 * passes[a][step];
      job_array[nj] = a;
      cur[a] = dst;
      ++nj;
    }
    dim3 grid(tiles, nj);
    k_onesweep<<<grid, kSwBlock, 0, st>>>(jobs, n, d_err);
    BITS_LAUNCH_CHECK("k_onesweep");
    (void)job_array;
  }
  return BITS_OK;
}

}  // namespace bits
