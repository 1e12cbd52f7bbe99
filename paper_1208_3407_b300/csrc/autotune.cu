// Method choice for BITS_METHOD_AUTO.
#include "count.cuh"

namespace bits {

int choose_count_method(const bits_db* db, uint32_t n) {
  (void)n;
  return db->has_rmi ? BITS_METHOD_RMI : BITS_METHOD_SEARCH;
}

}  // namespace bits
