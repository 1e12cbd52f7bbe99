// bits_sort_intervals_noalloc: the database sort without any device
// allocation, for callers that cannot call cudaMalloc.
//
// The radix sort of bits_build_db needs scratch memory (a ping-pong buffer
// per array, digit histograms, look-back words, tile tickets and an error
// word).  Here all of it lives in one file-scope device array of fixed size,
// so the call itself allocates nothing; the caller passes the input pairs and
// the two output arrays.  The array is part of the library image: every GPU
// that loads the library holds it (about 2.4 MB) until the process exits.
#include <mutex>
#include <vector>

#include "radix_sort.cuh"

namespace bits {
namespace {

constexpr uint32_t kMaxN = BITS_NOALLOC_MAX_INTERVALS;
constexpr size_t kTmpWords = kMaxN;               // one ping-pong buffer
constexpr size_t kHistWords = kRadixHistWords;    // 2 arrays x 4 passes x 256 digits + flag
constexpr size_t kTicketWords = 64;               // 2 x 4 used, padded to 256 B
constexpr size_t kErrWords = 64;                  // 1 used, padded to 256 B
constexpr size_t kStatusWords = radix_status_words_max(kMaxN) * 8;  // 2 arrays x 4 passes

constexpr size_t kOffTmpS = 0;
constexpr size_t kOffTmpE = kOffTmpS + kTmpWords;
constexpr size_t kOffHist = kOffTmpE + kTmpWords;
constexpr size_t kOffStatus = kOffHist + kHistWords;
constexpr size_t kOffTickets = kOffStatus + kStatusWords;
constexpr size_t kOffErr = kOffTickets + kTicketWords;
constexpr size_t kWords = kOffErr + kErrWords;

static_assert(kOffHist % 64 == 0 && kOffStatus % 64 == 0 && kOffTickets % 64 == 0 &&
                  kOffErr % 64 == 0,
              "every scratch region starts on a 256-byte boundary");

static __device__ __align__(256) uint32_t g_sort_scratch[kWords];

// Device address of g_sort_scratch, looked up once per device.  In host code
// the symbol names a host-side stand-in, so only this address may be handed
// to kernels or to cudaMemsetAsync.
std::mutex g_mu;
std::vector<uint32_t*> g_addr;

bits_status scratch_address(uint32_t** out) {
  int dev = 0;
  BITS_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_addr.size() <= dev) g_addr.resize(dev + 1, nullptr);
  if (!g_addr[dev]) {
    void* p = nullptr;
    BITS_CUDA_TRY(cudaGetSymbolAddress(&p, g_sort_scratch));
    g_addr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_addr[dev];
  return BITS_OK;
}

}  // namespace
}  // namespace bits

using namespace bits;

extern "C" bits_status bits_sort_intervals_noalloc(const uint32_t* d_b, uint64_t n,
                                                   uint32_t* d_bs, uint32_t* d_be,
                                                   void* stream) {
  if (n > kMaxN) {
    set_error("bits_sort_intervals_noalloc: n exceeds BITS_NOALLOC_MAX_INTERVALS (262144); "
              "use bits_build_db for larger databases");
    return BITS_EOVERFLOW;
  }
  if (n && (!d_b || !d_bs || !d_be)) {
    set_error("bits_sort_intervals_noalloc: NULL pointer");
    return BITS_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(d_b) % 8 || reinterpret_cast<uintptr_t>(d_bs) % 4 ||
      reinterpret_cast<uintptr_t>(d_be) % 4) {
    set_error("bits_sort_intervals_noalloc: misaligned pointer (pairs 8 B, outputs 4 B)");
    return BITS_EINVAL;
  }
  if (n == 0) return BITS_OK;
  uint32_t* base = nullptr;
  bits_status s = scratch_address(&base);
  if (s != BITS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The array keeps the previous call's contents; only the error word needs
  // clearing here (the sort zeroes its histograms, look-back words and
  // tickets itself).
  uint32_t* err = base + kOffErr;
  BITS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(uint32_t), st));
  RadixScratch ws{};
  ws.tmp_s = base + kOffTmpS;
  ws.tmp_e = base + kOffTmpE;
  ws.hist = base + kOffHist;
  ws.status = base + kOffStatus;
  ws.tickets = base + kOffTickets;
  s = radix_sort_intervals(reinterpret_cast<const uint2*>(d_b), (uint32_t)n, d_bs, d_be, err, ws,
                           st);
  if (s != BITS_OK) return s;
  uint32_t h = 0;
  BITS_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  BITS_CUDA_TRY(cudaStreamSynchronize(st));
  if (h & DEV_ERR_INTERNAL) {
    set_error("bits_sort_intervals_noalloc: a device-side consistency check failed (sort "
              "scatter index out of range)");
    return BITS_EINTERNAL;
  }
  if (h & DEV_ERR_TIMEOUT) {
    set_error("bits_sort_intervals_noalloc: a bounded device-side wait timed out");
    return BITS_ETIMEOUT;
  }
  return BITS_OK;
}
