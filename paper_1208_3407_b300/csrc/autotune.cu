// Method choice for BITS_METHOD_AUTO.
//
// The first AUTO count of a size class -- (device, ceil log2 |A|, ceil log2
// |B|, learned index built or not, per-query counts wanted or not) -- times
// every method the database has (plain search, learned index, merge path
// when the query set is at least 1/16 of the database) on the caller's own
// inputs with CUDA events: batches of back-to-back calls lasting about half
// a millisecond, three rounds alternating the methods, fastest batch per
// method; the fastest method wins.  Later calls of the class reuse the
// choice.  When BITS_AUTOTUNE_CACHE names a file, choices
// are read from it at first use and appended to it as they are made.  Under
// stream capture no timing is possible, so the learned index (if built) or
// the plain search is used without tuning.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "count.cuh"
#include "mergepath.cuh"
#include "rmi.cuh"

namespace bits {
namespace {

using Key = std::tuple<std::string, int, int, int>;
std::mutex g_mu;
std::map<Key, int> g_choice;
bool g_loaded = false;

int ceil_log2(uint64_t x) {
  int k = 0;
  while ((1ull << k) < x) ++k;
  return k;
}

std::string device_name() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p{};
  cudaGetDeviceProperties(&p, dev);
  std::string s(p.name);
  for (char& c : s)
    if (c == ' ') c = '_';
  return s;
}

void load_cache() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = std::getenv("BITS_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char name[256];
  int la, lb, rmi, m;
  while (std::fscanf(f, "%255s %d %d %d %d", name, &la, &lb, &rmi, &m) == 5)
    g_choice[Key(name, la, lb, rmi)] = m;
  std::fclose(f);
}

void save_choice(const Key& k, int m) {
  const char* path = std::getenv("BITS_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %d\n", std::get<0>(k).c_str(), std::get<1>(k), std::get<2>(k),
               std::get<3>(k), m);
  std::fclose(f);
}

bits_status run_method(const bits_db* db, int m, const uint32_t* d_a, uint32_t n,
                       uint32_t* d_counts, uint64_t* d_total, cudaStream_t st) {
  if (m == BITS_METHOD_RMI) return launch_count_rmi(db, d_a, n, d_counts, d_total, st);
  if (m == BITS_METHOD_MERGEPATH) return launch_count_mergepath(db, d_a, n, d_counts, d_total, st);
  return launch_count_search(db, d_a, n, d_counts, d_total, st);
}

// Merge path streams all of B per call, so it is only a candidate when the
// query set is at least 1/16 of the database.
bool mergepath_candidate(const bits_db* db, uint32_t n) {
  return n < (1u << 31) && (uint64_t)n * 16 >= db->n;
}

}  // namespace

int choose_count_method(const bits_db* db, uint32_t n) {
  const int fallback = db->has_rmi ? BITS_METHOD_RMI : BITS_METHOD_SEARCH;
  std::lock_guard<std::mutex> lk(g_mu);
  load_cache();
  auto it = g_choice.find(Key(device_name(), ceil_log2(n), ceil_log2(db->n),
                             (db->has_rmi ? 1 : 0) | 2));
  return it == g_choice.end() ? fallback : it->second;
}

bits_status autotune_count(const bits_db* db, const uint32_t* d_a, uint32_t n,
                           uint32_t* d_counts, uint64_t* d_total, cudaStream_t st, int* method) {
  const Key key(device_name(), ceil_log2(n), ceil_log2(db->n),
                (db->has_rmi ? 1 : 0) | (d_counts ? 2 : 0));
  std::vector<int> cands = {BITS_METHOD_SEARCH};
  if (db->has_rmi) cands.push_back(BITS_METHOD_RMI);
  if (mergepath_candidate(db, n)) cands.push_back(BITS_METHOD_MERGEPATH);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache();
    auto it = g_choice.find(key);
    if (it != g_choice.end()) {
      *method = it->second;
      return BITS_OK;
    }
  }
  *method = db->has_rmi ? BITS_METHOD_RMI : BITS_METHOD_SEARCH;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  BITS_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone || cands.size() < 2 || n == 0) return BITS_OK;

  // Each candidate is timed on R back-to-back calls between one pair of
  // events, R chosen so that a batch lasts about half a millisecond, over
  // three rounds that alternate the candidates; its fastest batch counts.
  // Event timestamps advance in steps of about 2 us, so single calls on a
  // small sample are too short to tell the methods apart.
  cudaEvent_t e0, e1;
  BITS_CUDA_TRY(cudaEventCreate(&e0));
  BITS_CUDA_TRY(cudaEventCreate(&e1));
  auto batch = [&](int m, int reps, float* ms) -> bits_status {
    BITS_CUDA_TRY(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) {
      bits_status s = run_method(db, m, d_a, n, d_counts, d_total, st);
      if (s != BITS_OK) return s;
    }
    BITS_CUDA_TRY(cudaEventRecord(e1, st));
    BITS_CUDA_TRY(cudaEventSynchronize(e1));
    BITS_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    return BITS_OK;
  };
  float single = 0.f;
  for (int m : cands) {
    float ms = 0.f;
    bits_status s = batch(m, 2, &ms);  // warm-up, and the size of one call
    if (s != BITS_OK) return s;
    single = std::max(single, ms / 2.f);
  }
  const int reps = std::max(1, std::min(64, (int)(0.5f / std::max(single, 1e-3f)) + 1));
  std::vector<float> best_ms(cands.size(), 1e30f);
  for (int round = 0; round < 3; ++round) {
    for (size_t c = 0; c < cands.size(); ++c) {
      float ms = 0.f;
      bits_status s = batch(cands[c], reps, &ms);
      if (s != BITS_OK) return s;
      best_ms[c] = std::min(best_ms[c], ms);
    }
  }
  int best_m = cands[0];
  float best = best_ms[0];
  for (size_t c = 1; c < cands.size(); ++c)
    if (best_ms[c] < best) {
      best = best_ms[c];
      best_m = cands[c];
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *method = best_m;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_choice.emplace(key, best_m).second) save_choice(key, best_m);
  return BITS_OK;
}

}  // namespace bits
