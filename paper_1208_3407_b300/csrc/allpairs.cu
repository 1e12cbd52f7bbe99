#include "allpairs.cuh"

namespace bits {

bits_status run_count_matrix(const bits_db* const*, uint32_t, const uint32_t* const*,
                             const uint64_t*, uint32_t, uint64_t*, cudaStream_t) {
  set_error("bits_count_matrix: not built yet");
  return BITS_ENOTIMPL;
}

}  // namespace bits
