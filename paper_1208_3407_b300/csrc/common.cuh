// Shared definitions of the BITS CUDA library (device + host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "../../include/bits.h"

namespace bits {

// Bits OR-ed into a database's device error word.
enum : uint32_t {
  DEV_ERR_INVALID = 1u,   // an interval violated the input rules
  DEV_ERR_TIMEOUT = 2u,   // a bounded spin-wait gave up
  DEV_ERR_INTERNAL = 4u,  // an internal consistency check failed (index out of range)
};

// Iterations a spin-wait may take (each sleeps ~100-200 ns) before it gives
// up and reports DEV_ERR_TIMEOUT: about one second of waiting.
constexpr uint32_t kSpinLimit = 1u << 23;

constexpr uint32_t kU32Max = 0xFFFFFFFFu;

// Host helpers (defined in capi.cu).
void set_error(const std::string& msg);
void count_launch(uint32_t k = 1);
void uncount_launch(uint64_t k);
int sm_count();
// Resident CTAs per SM of `kernel` with `block` threads and `smem` bytes of
// dynamic shared memory on the current device (at least 1; at most `cap`
// when cap > 0).  The kernel's dynamic shared-memory limit on the device is
// raised to `smem` if it is lower (it never drops, so earlier launch sizes
// stay valid); with cap > 0 the shared-memory carveout is fitted to that
// many CTAs so the rest of the SM's on-chip memory stays L1.  Both are
// per-device settings, kept per (device, kernel) under a lock.
int kernel_blocks_per_sm(const void* kernel, int block, size_t smem, int cap = 0);
bits_status cuda_status(cudaError_t e, const char* what);
// Device memory from the library's stream-ordered pool, one per device,
// created at first use: database blocks and every temporary (sort buffers,
// merge-path keys, enumeration counts, staging of host buffers).  Freed
// blocks return to the pool (pool_free, or cudaFree for a database) and up
// to kPoolKeepBytes stay reserved across synchronisations, so repeated
// calls and rebuilt databases make no driver allocation.
constexpr uint64_t kPoolKeepBytes = 4ull << 30;
bits_status pool_alloc(void** p, size_t bytes, cudaStream_t st);
inline void pool_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

#define BITS_CUDA_TRY(expr)                                         \
  do {                                                              \
    cudaError_t _e = (expr);                                        \
    if (_e != cudaSuccess) return ::bits::cuda_status(_e, #expr);   \
  } while (0)

#define BITS_LAUNCH_CHECK(what)                                     \
  do {                                                              \
    ::bits::count_launch();                                         \
    cudaError_t _e = cudaGetLastError();                            \
    if (_e != cudaSuccess) return ::bits::cuda_status(_e, what);    \
  } while (0)

// Launch configuration of a programmatic dependent launch: the kernel may
// start while the kernel before it in the stream drains, and must execute
// griddepcontrol.wait before it touches what that kernel writes.
inline void pdl_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, dim3 grid, dim3 block,
                       size_t smem, cudaStream_t st) {
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void set_dev_error(uint32_t* err, uint32_t bit) {
  if (err) atomicOr(err, bit);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// 64-bit block sum; result valid in thread 0.  `red` holds >= 32 entries.
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                            unsigned long long* red) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  const unsigned w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane_id() == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane_id() < nw ? red[lane_id()] : 0ull;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  }
  return v;
}

}  // namespace bits
