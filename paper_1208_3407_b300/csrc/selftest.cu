// bits_selftest_wait: exercises the bounded device-side wait.
//
// Every spin-wait in the library (the radix sort's decoupled look-back) is a
// volatile load of a device word, a short sleep, and an iteration cap after
// which the kernel records DEV_ERR_TIMEOUT and returns instead of hanging.
// This entry point runs that pattern on a word nothing ever sets, so the cap
// always runs out: the call must return BITS_ETIMEOUT and leave the context
// usable for the calls that follow.
#include "common.cuh"

namespace bits {
namespace {

__global__ void k_selftest_wait(const uint32_t* word, uint32_t limit, uint32_t* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t spins = 0;
  while (*(volatile const uint32_t*)word == 0u) {
    if (++spins > limit) {
      set_dev_error(err, DEV_ERR_TIMEOUT);
      return;
    }
    __nanosleep(64);
  }
}

}  // namespace
}  // namespace bits

using namespace bits;

extern "C" bits_status bits_selftest_wait(uint32_t spin_limit, void* stream) {
  if (spin_limit == 0 || spin_limit > kSpinLimit) {
    set_error("bits_selftest_wait: spin_limit must be in [1, 2^23]");
    return BITS_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* d = nullptr;
  {
    const bits_status as = pool_alloc(reinterpret_cast<void**>(&d), 2 * sizeof(uint32_t), st);
    if (as != BITS_OK) return as;
  }
  BITS_CUDA_TRY(cudaMemsetAsync(d, 0, 2 * sizeof(uint32_t), st));
  k_selftest_wait<<<1, 32, 0, st>>>(d, spin_limit, d + 1);
  count_launch();
  uint32_t h = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  pool_free(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "bits_selftest_wait");
  if (h & DEV_ERR_TIMEOUT) {
    set_error("bits_selftest_wait: the bounded wait ran out, as it must");
    return BITS_ETIMEOUT;
  }
  return BITS_OK;
}
