// bits_probe_random_reads: the rate at which this GPU serves random 64-byte
// node reads from DRAM.  Built into its own library, libbits_probe.so (a
// measurement aid for the benchmark, not part of the method).
//
// Every search kernel here reads one 64-byte node per level of the 16-ary
// tree, loaded by a quad of lanes (16 bytes each) with a 64-byte line fill.
// On a database much larger than L2 the level-0 nodes come from DRAM at
// random, and the rate of such reads, not the byte bandwidth, limits the
// kernels: independent random 64-byte reads over a buffer far beyond L2
// reach about a third of the copy bandwidth (the tree's interleaved node
// pairs let the counts go somewhat beyond that rate).
// This probe issues exactly that access -- quads reading uniformly random
// nodes of a buffer, four independent accesses in flight per quad -- and
// times it with CUDA events, so the search kernels can be set against the
// same hardware limit.  Access kinds 2 and 3 read both 64-byte halves of one
// random 128-byte line, as a query does whose two searches (starts and ends)
// meet in one interleaved node pair: kind 2 with two loads, kind 3 with one
// load instruction of eight lanes.  The rate follows the number of load
// requests, not the bytes: kind 3 runs at the kind-1 rate, kind 2 at half.
#include "common.cuh"
#include "../../include/bits_probe.h"

namespace bits {
namespace {

constexpr int kProbeBlock = 512;
constexpr int kProbeInFlight = 4;

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  // Murmur3's 32-bit finaliser: spreads the node index over the buffer.
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

// One random access per (group, k): kind 1, a 64-byte node loaded by a quad
// (16 bytes a lane); kind 2, both 64-byte halves of one random 128-byte
// line loaded by a quad as two node loads (the access of the quad descent
// when a query's two searches meet in one interleaved node pair); kind 3,
// the same line loaded by an octet with ONE instruction (the octet descent).
// An octet is two quads, so it makes twice a quad's accesses per round and
// every kind makes the same number of accesses per round of the grid.
template <int kKind>
__global__ void __launch_bounds__(kProbeBlock)
k_probe_random(const uint4* __restrict__ buf, uint64_t n_units, uint32_t iters,
               unsigned long long* __restrict__ sink) {
  constexpr uint32_t kLanes = kKind == 3 ? 8u : 4u;          // lanes per access
  constexpr uint32_t kUnit = kKind == 1 ? 4u : 8u;           // 16-byte words per access
  constexpr int kFlight = kKind == 3 ? 2 * kProbeInFlight : kProbeInFlight;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t grp = tid / kLanes, sub = tid % kLanes;
  uint32_t acc = 0;
  for (uint32_t it = 0; it < iters; ++it) {
    uint4 v[kFlight], w[kFlight];
#pragma unroll
    for (int k = 0; k < kFlight; ++k) {
      const uint32_t h = mix32(grp * 0x9E3779B9u + (it * kFlight + k) * 0x632BE5ABu);
      const uint64_t unit = ((uint64_t)h * n_units) >> 32;  // < n_units
      const uint4* p = buf + unit * kUnit + sub;
      asm volatile("ld.global.nc.L2::64B.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(v[k].x), "=r"(v[k].y), "=r"(v[k].z), "=r"(v[k].w)
                   : "l"(p));
      if (kKind == 2) {
        asm volatile("ld.global.nc.L2::64B.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(w[k].x), "=r"(w[k].y), "=r"(w[k].z), "=r"(w[k].w)
                     : "l"(p + 4));
      } else {
        w[k] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
#pragma unroll
    for (int k = 0; k < kFlight; ++k) acc += v[k].x ^ v[k].w ^ w[k].y;
  }
  // Keeps the loads alive: the result depends on the data read, so the
  // compiler cannot drop them (taken with probability 2^-32 per thread).
  if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);
}

}  // namespace
}  // namespace bits

using namespace bits;

extern "C" bits_status bits_probe_random_reads(const void* d_buf, uint64_t bytes,
                                               uint64_t n_reads, int32_t access_kind,
                                               double* h_accesses_per_s, void* stream) {
  if (!d_buf || !h_accesses_per_s) {
    set_error("bits_probe_random_reads: NULL argument");
    return BITS_EINVAL;
  }
  if (access_kind < 1 || access_kind > 3) {
    set_error("bits_probe_random_reads: access_kind must be 1, 2 or 3");
    return BITS_EINVAL;
  }
  const uint64_t unit = access_kind == 1 ? 64ull : 128ull;
  if (bytes < unit || bytes % unit || bytes / unit >= (1ull << 32) ||
      reinterpret_cast<uintptr_t>(d_buf) % unit) {
    set_error("bits_probe_random_reads: the buffer must be aligned to and hold 1 .. 2^32 - 1 "
              "whole accesses (64 bytes for access kind 1, else 128)");
    return BITS_EINVAL;
  }
  if (n_reads == 0 || n_reads > (1ull << 34)) {
    set_error("bits_probe_random_reads: n_reads must be in [1, 2^34]");
    return BITS_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t blocks = 2u * (uint32_t)sm_count();
  const uint64_t quads = (uint64_t)blocks * kProbeBlock / 4u;
  const uint64_t per_iter = quads * kProbeInFlight;
  const uint32_t iters = (uint32_t)std::max<uint64_t>(1, (n_reads + per_iter - 1) / per_iter);
  unsigned long long* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  {
    const bits_status as = pool_alloc(reinterpret_cast<void**>(&sink), sizeof(*sink), st);
    if (as != BITS_OK) return as;
  }
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    const uint4* b = static_cast<const uint4*>(d_buf);
    if (access_kind == 3)
      k_probe_random<3><<<blocks, kProbeBlock, 0, st>>>(b, bytes / unit, iters, sink);
    else if (access_kind == 2)
      k_probe_random<2><<<blocks, kProbeBlock, 0, st>>>(b, bytes / unit, iters, sink);
    else
      k_probe_random<1><<<blocks, kProbeBlock, 0, st>>>(b, bytes / unit, iters, sink);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  pool_free(sink, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_status(e, "bits_probe_random_reads");
  *h_accesses_per_s = ms > 0.f ? (double)iters * (double)per_iter / (ms * 1e-3) : 0.0;
  return BITS_OK;
}
