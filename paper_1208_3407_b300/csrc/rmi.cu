#include "rmi.cuh"

namespace bits {

bits_status rmi_build(const uint32_t*, uint32_t, bits_rmi&, cudaStream_t) {
  set_error("learned index: not built yet");
  return BITS_ENOTIMPL;
}

bits_status launch_count_rmi(const bits_db*, const uint32_t*, uint32_t, uint32_t*, uint64_t*,
                             cudaStream_t) {
  set_error("learned index: not built yet");
  return BITS_ENOTIMPL;
}

}  // namespace bits
