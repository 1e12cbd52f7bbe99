// bits_count_host: Algorithm 2's counting loop over queries and counts that
// live in host memory, end to end in one call.
//
// Page-locked host buffers (cudaHostAlloc, cudaMallocHost, cudaHostRegister)
// are read and written in place by the count kernel over the bus: each
// thread's 8-byte query load and 4-byte count store cross it directly, so
// the transfer overlaps the searches and no staging copy or device buffer is
// needed.  A pageable buffer is never handed to a kernel: it is staged
// through a stream-ordered device buffer with cudaMemcpyAsync.  The 64-bit
// total is added up in a stream-ordered device word of its own per call
// (so calls on different streams do not share it) and copied back.  Both
// come from the library's stream-ordered memory pool (pool_alloc).

#include "count.cuh"
#include "db.cuh"
#include "mergepath.cuh"
#include "rmi.cuh"

namespace bits {
namespace {

// Device address of a host range the GPU can reach in place, or nullptr when
// the range is not page-locked host memory.  The first and the last byte
// must both belong to page-locked host memory at consecutive device
// addresses; anything else is staged.
bits_status device_alias(const void* p, size_t bytes, const void** dev, const char* what) {
  *dev = nullptr;
  if (!p || bytes == 0) return BITS_OK;
  cudaPointerAttributes a0{}, a1{};
  cudaError_t e0 = cudaPointerGetAttributes(&a0, p);
  if (e0 != cudaSuccess) {
    cudaGetLastError();
    return BITS_OK;
  }
  if (a0.type == cudaMemoryTypeDevice || a0.type == cudaMemoryTypeManaged) {
    set_error(std::string("bits_count_host: ") + what +
              " is device or managed memory; use bits_count for device buffers");
    return BITS_EINVAL;
  }
  if (a0.type != cudaMemoryTypeHost || !a0.devicePointer) return BITS_OK;
  const char* last = static_cast<const char*>(p) + (bytes - 1);
  cudaError_t e1 = cudaPointerGetAttributes(&a1, last);
  if (e1 != cudaSuccess) {
    cudaGetLastError();
    return BITS_OK;
  }
  if (a1.type != cudaMemoryTypeHost || !a1.devicePointer ||
      static_cast<const char*>(a1.devicePointer) - static_cast<const char*>(a0.devicePointer) !=
          (ptrdiff_t)(bytes - 1))
    return BITS_OK;
  *dev = a0.devicePointer;
  return BITS_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace bits

using namespace bits;

extern "C" bits_status bits_count_host(const bits_db* db, int32_t method, const uint32_t* h_a,
                                       uint64_t n, uint32_t* h_counts, uint64_t* h_total,
                                       void* stream) {
  if (!db || !h_total || (n && !h_a)) {
    set_error("bits_count_host: NULL argument");
    return BITS_EINVAL;
  }
  if (n >= (1ull << 32)) {
    set_error("bits_count_host: at most 2^32 - 1 queries per call");
    return BITS_EOVERFLOW;
  }
  if (reinterpret_cast<uintptr_t>(h_a) % 8 || reinterpret_cast<uintptr_t>(h_counts) % 4 ||
      reinterpret_cast<uintptr_t>(h_total) % 8) {
    set_error("bits_count_host: misaligned pointer (queries 8 B, counts 4 B, total 8 B)");
    return BITS_EINVAL;
  }
  if (method < BITS_METHOD_AUTO || method > BITS_METHOD_MERGEPATH) {
    set_error("bits_count_host: unknown method");
    return BITS_EINVAL;
  }
  if (method == BITS_METHOD_RMI && !db->has_rmi) {
    set_error("bits_count_host: database was built without a learned index");
    return BITS_ENOTIMPL;
  }
  // Method (for AUTO), top and CTA size as recorded for this size class (the
  // host-buffer path itself never times candidates).
  const TuneCount tuned = count_params(db, method, (uint32_t)n, h_counts != nullptr);
  method = tuned.method;
  int cur = 0;
  BITS_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != db->device) {
    set_error("bits_count_host: the database belongs to another device than the current one");
    return BITS_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t a_bytes = sizeof(uint64_t) * n, c_bytes = sizeof(uint32_t) * n;

  // Queries and counts: in place when page-locked, else staged.  The total
  // is always copied back (into page-locked or pageable memory alike);
  // its pointer is only checked not to be device memory.
  const void* a_alias = nullptr;
  const void* c_alias = nullptr;
  const void* t_alias = nullptr;
  bits_status s = device_alias(h_a, a_bytes, &a_alias, "h_a");
  if (s == BITS_OK) s = device_alias(h_counts, c_bytes, &c_alias, "h_counts");
  if (s == BITS_OK) s = device_alias(h_total, sizeof(uint64_t), &t_alias, "h_total");
  if (s != BITS_OK) return s;
  // Merge path sorts the queries on the device and streams them several
  // times: it always works on device copies.
  const bool stage_a = n && (!a_alias || method == BITS_METHOD_MERGEPATH);
  const bool stage_c = n && h_counts && (!c_alias || method == BITS_METHOD_MERGEPATH);
  // One stream-ordered block per call: the 64-bit total the kernel adds
  // into, then the staged queries and counts, if any.
  const size_t off_a = 256;
  const size_t off_c = off_a + (stage_a ? align256(a_bytes) : 0);
  const size_t bytes = off_c + (stage_c ? align256(c_bytes) : 0);
  char* buf = nullptr;
  s = pool_alloc(reinterpret_cast<void**>(&buf), bytes, st);
  if (s != BITS_OK) return s;
  auto done = [&](bits_status r) {
    pool_free(buf, st);
    return r;
  };
  uint64_t* d_total = reinterpret_cast<uint64_t*>(buf);
  const uint32_t* d_a = static_cast<const uint32_t*>(a_alias);
  uint32_t* d_c = h_counts ? static_cast<uint32_t*>(const_cast<void*>(c_alias)) : nullptr;
  if (stage_a) {
    d_a = reinterpret_cast<const uint32_t*>(buf + off_a);
    cudaError_t e = cudaMemcpyAsync(buf + off_a, h_a, a_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return done(cuda_status(e, "cudaMemcpyAsync(queries)"));
  }
  if (stage_c) d_c = reinterpret_cast<uint32_t*>(buf + off_c);

  s = launch_count_tuned(db, tuned, d_a, (uint32_t)n, d_c, d_total, st);
  if (s != BITS_OK) return done(s);
  if (stage_c) {
    cudaError_t e = cudaMemcpyAsync(h_counts, d_c, c_bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return done(cuda_status(e, "cudaMemcpyAsync(counts)"));
  }
  cudaError_t e = cudaMemcpyAsync(h_total, d_total, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return done(cuda_status(e, "cudaMemcpyAsync(total)"));
  return done(BITS_OK);
}
