#include "mc.cuh"

namespace bits {

bits_status run_mc(bits_db*, int, const uint32_t*, uint32_t, const uint32_t*, const uint32_t*,
                   uint32_t, uint64_t, uint32_t, uint32_t, uint64_t*, uint64_t*, uint64_t*,
                   double*, cudaStream_t) {
  set_error("bits_mc: not built yet");
  return BITS_ENOTIMPL;
}

void release_mc_graphs(bits_db* db) { db->mc_graphs.clear(); }

}  // namespace bits
