#include "mergepath.cuh"

namespace bits {

bits_status launch_count_mergepath(const bits_db*, const uint32_t*, uint32_t, uint32_t*,
                                   uint64_t*, cudaStream_t) {
  set_error("merge-path count: not built yet");
  return BITS_ENOTIMPL;
}

}  // namespace bits
