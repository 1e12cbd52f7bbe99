// The autotuner: launch parameters per size class, chosen by timing.
//
// What it tunes (none of it changes a result; see tune.cuh):
//   * bits_count: the method (plain search, learned index, merge path when
//     the query set is at least 1/16 of the database), the shared-memory top
//     of the plain search (the database's default top level or one or two
//     levels above it: a smaller top, one more tree level read from memory)
//     and the threads per CTA of the search kernels (256 or 512);
//   * bits_mc: shuffles and intervals per work unit and the top (mc.cu);
//   * bits_count_matrix: queries per work unit (allpairs.cu).
// A size class is (device, ceil log2 of the queries, ceil log2 of the
// database, learned index built or not, per-query counts wanted or not).
// The first call of a class that is neither pinned by bits_set_tuning nor
// under stream capture times every candidate on the caller's own inputs
// with CUDA events -- batches of back-to-back calls lasting about half a
// millisecond, three rounds alternating the candidates, fastest batch per
// candidate -- and records the fastest overall (the AUTO method) and the
// fastest of each method (calls that name their method).  Later calls of
// the class reuse the record.  When BITS_AUTOTUNE_CACHE names a file,
// records are read from it at first use and appended to it as they are
// made, one line each:
//     <device> <kind> <log2 queries> <log2 database> <flags> <values...>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "count.cuh"
#include "mergepath.cuh"
#include "rmi.cuh"
#include "tune.cuh"

namespace bits {
namespace {

using Key = std::tuple<std::string, std::string, int, int, int>;
std::mutex g_mu;
std::map<Key, std::vector<int>> g_cache;
bool g_loaded = false;
thread_local bits_tuning g_pin = {-1, 0, 0, 0, 0};

std::string device_name() {
  static std::mutex mu;
  static std::vector<std::string> names;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if ((int)names.size() <= dev) names.resize(dev + 1);
  if (names[dev].empty()) {
    cudaDeviceProp p{};
    cudaGetDeviceProperties(&p, dev);
    std::string s(p.name);
    for (char& c : s)
      if (c == ' ') c = '_';
    names[dev] = s.empty() ? "gpu" : s;
  }
  return names[dev];
}

void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = std::getenv("BITS_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof(line), f)) {
    std::istringstream in(line);
    std::string dev, kind;
    int la, lb, fl;
    if (!(in >> dev >> kind >> la >> lb >> fl)) continue;
    std::vector<int> vals;
    int v;
    while (in >> v) vals.push_back(v);
    if (!vals.empty()) g_cache[Key(dev, kind, la, lb, fl)] = vals;
  }
  std::fclose(f);
}

void save_locked(const Key& k, const std::vector<int>& vals) {
  const char* path = std::getenv("BITS_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %s %d %d %d", std::get<0>(k).c_str(), std::get<1>(k).c_str(),
               std::get<2>(k), std::get<3>(k), std::get<4>(k));
  for (int v : vals) std::fprintf(f, " %d", v);
  std::fprintf(f, "\n");
  std::fclose(f);
}

// Merge path streams all of B per call, so it is only a candidate when the
// query set is at least 1/16 of the database.
bool mergepath_candidate(const bits_db* db, uint32_t n) {
  return n < (1u << 31) && (uint64_t)n * 16 >= db->n;
}

int count_flags(const bits_db* db, bool counts, int method) {
  return (db->has_rmi ? 1 : 0) | (counts ? 2 : 0) | (method << 2);
}

int max_raise(const bits_db* db) { return db->plan.Tmax - db->plan.J; }

bool count_pinned() { return g_pin.top_raise >= 0 || g_pin.block > 0; }

}  // namespace

const bits_tuning& pinned_tuning() { return g_pin; }

int ceil_log2_u64(uint64_t x) {
  int k = 0;
  while ((1ull << k) < x && k < 63) ++k;
  return k;
}

bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;  // unknown: do not time anything
  }
  return cs != cudaStreamCaptureStatusNone;
}

bool tune_lookup(const char* kind, int la, int lb, int flags, std::vector<int>* vals) {
  const Key k(device_name(), kind, la, lb, flags);
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  auto it = g_cache.find(k);
  if (it == g_cache.end()) return false;
  if (vals) *vals = it->second;
  return true;
}

void tune_store(const char* kind, int la, int lb, int flags, const std::vector<int>& vals) {
  const Key k(device_name(), kind, la, lb, flags);
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  if (g_cache.emplace(k, vals).second) save_locked(k, vals);
}

TuneCount count_params(const bits_db* db, int method, uint32_t n, bool counts) {
  TuneCount t;
  // AUTO without a record (parameters pinned, stream capture) takes the
  // plain search, the faster form on every shape measured.
  t.method = method == BITS_METHOD_AUTO ? BITS_METHOD_SEARCH : method;
  std::vector<int> v;
  if (tune_lookup("count", ceil_log2_u64(n), ceil_log2_u64(db->n),
                  count_flags(db, counts, method), &v) &&
      v.size() == 3) {
    t.method = v[0];
    t.raise = v[1];
    t.block = v[2];
  }
  if (t.method == BITS_METHOD_RMI && !db->has_rmi) t.method = BITS_METHOD_SEARCH;
  if (g_pin.top_raise >= 0) t.raise = g_pin.top_raise;
  if (g_pin.block > 0) t.block = g_pin.block;
  t.raise = std::max(0, std::min(t.raise, max_raise(db)));
  if (t.block != 256) t.block = 512;
  return t;
}

bits_status launch_count_tuned(const bits_db* db, const TuneCount& t, const uint32_t* d_a,
                               uint32_t n, uint32_t* d_counts, uint64_t* d_total,
                               cudaStream_t st) {
  switch (t.method) {
    case BITS_METHOD_RMI:
      return launch_count_rmi(db, d_a, n, d_counts, d_total, st, &t);
    case BITS_METHOD_MERGEPATH:
      return launch_count_mergepath(db, d_a, n, d_counts, d_total, st);
    default:
      return launch_count_search(db, d_a, n, d_counts, d_total, st, &t);
  }
}

bits_status autotune_count(const bits_db* db, const uint32_t* d_a, uint32_t n,
                           uint32_t* d_counts, uint64_t* d_total, cudaStream_t st, int method,
                           TuneCount* out) {
  const bool counts = d_counts != nullptr;
  const int la = ceil_log2_u64(n), lb = ceil_log2_u64(db->n);
  *out = count_params(db, method, n, counts);
  if (n == 0 || count_pinned() ||
      tune_lookup("count", la, lb, count_flags(db, counts, method), nullptr) ||
      stream_capturing(st))
    return BITS_OK;

  std::vector<TuneCount> cands;
  for (int r = 0; r <= max_raise(db); ++r)
    for (int b : kCountBlocks) cands.push_back(TuneCount{BITS_METHOD_SEARCH, r, b});
  if (db->has_rmi)
    for (int b : kCountBlocks) cands.push_back(TuneCount{BITS_METHOD_RMI, 0, b});
  if (mergepath_candidate(db, n)) cands.push_back(TuneCount{BITS_METHOD_MERGEPATH, 0, 512});

  // Each candidate is timed on R back-to-back calls between one pair of
  // events, R chosen so that a batch lasts about half a millisecond, over
  // three rounds that alternate the candidates; its fastest batch counts.
  // Event timestamps advance in steps of about 2 us, so single calls on a
  // small input are too short to tell the candidates apart.
  cudaEvent_t e0, e1;
  BITS_CUDA_TRY(cudaEventCreate(&e0));
  BITS_CUDA_TRY(cudaEventCreate(&e1));
  auto batch = [&](const TuneCount& c, int reps, float* ms) -> bits_status {
    BITS_CUDA_TRY(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) {
      bits_status s = launch_count_tuned(db, c, d_a, n, d_counts, d_total, st);
      if (s != BITS_OK) return s;
    }
    BITS_CUDA_TRY(cudaEventRecord(e1, st));
    BITS_CUDA_TRY(cudaEventSynchronize(e1));
    BITS_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    return BITS_OK;
  };
  auto finish = [&](bits_status s) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
  };
  float single = 0.f;
  for (const TuneCount& c : cands) {
    float ms = 0.f;
    bits_status s = batch(c, 2, &ms);  // warm-up, and the size of one call
    if (s != BITS_OK) return finish(s);
    single = std::max(single, ms / 2.f);
  }
  const int reps = std::max(1, std::min(64, (int)(0.5f / std::max(single, 1e-3f)) + 1));
  std::vector<float> best_ms(cands.size(), 1e30f);
  for (int round = 0; round < 3; ++round)
    for (size_t c = 0; c < cands.size(); ++c) {
      float ms = 0.f;
      bits_status s = batch(cands[c], reps, &ms);
      if (s != BITS_OK) return finish(s);
      best_ms[c] = std::min(best_ms[c], ms);
    }
  // Record the fastest of each method, and for AUTO the fastest plain
  // search unless another method beats it by at least 5 %: on short calls
  // the batches differ by little more than their timing noise, and a
  // learned index chosen by noise costs more per query wherever the choice
  // is reused at larger sizes (the all-pairs kernel applies it to every
  // query set).
  int best_of[4] = {-1, -1, -1, -1};
  for (size_t c = 0; c < cands.size(); ++c) {
    int& b = best_of[cands[c].method];
    if (b < 0 || best_ms[c] < best_ms[b]) b = (int)c;
  }
  int best_auto = best_of[BITS_METHOD_SEARCH];
  for (int m : {(int)BITS_METHOD_RMI, (int)BITS_METHOD_MERGEPATH})
    if (best_of[m] >= 0 && (best_auto < 0 || best_ms[best_of[m]] < 0.95f * best_ms[best_auto]))
      best_auto = best_of[m];
  best_of[BITS_METHOD_AUTO] = best_auto;
  for (int m : {(int)BITS_METHOD_AUTO, (int)BITS_METHOD_SEARCH, (int)BITS_METHOD_RMI,
                (int)BITS_METHOD_MERGEPATH}) {
    const int best = best_of[m];
    if (best >= 0)
      tune_store("count", la, lb, count_flags(db, counts, m),
                 {cands[best].method, cands[best].raise, cands[best].block});
  }
  *out = count_params(db, method, n, counts);
  return finish(BITS_OK);
}

TuneMc mc_params(const bits_db* db, int method, uint32_t n, bool* tuned) {
  TuneMc t;
  std::vector<int> v;
  const bool have = tune_lookup("mc", ceil_log2_u64(n), ceil_log2_u64(db->n), method, &v) &&
                    v.size() == 3;
  if (have) {
    t.shuffles = v[0];
    t.chunk = v[1];
    t.raise = v[2];
  }
  if (tuned) *tuned = have;
  if (g_pin.mc_shuffles > 0) {
    t.shuffles = g_pin.mc_shuffles;
    t.chunk = g_pin.mc_chunk;
  }
  if (g_pin.top_raise >= 0) t.raise = g_pin.top_raise;
  if (method == BITS_METHOD_RMI) t.raise = 0;
  t.raise = std::max(0, std::min(t.raise, max_raise(db)));
  return t;
}

void mc_record(const bits_db* db, int method, uint32_t n, const TuneMc& t) {
  tune_store("mc", ceil_log2_u64(n), ceil_log2_u64(db->n), method, {t.shuffles, t.chunk, t.raise});
}

bool mc_pinned() { return g_pin.mc_shuffles > 0 || g_pin.top_raise >= 0; }

int ap_chunk_params(uint64_t total_queries, uint64_t total_db, uint32_t n_db, uint32_t n_sets,
                    bool* tuned, const char* kind) {
  if (tuned) *tuned = false;
  if (g_pin.ap_chunk > 0) {
    if (tuned) *tuned = true;
    return g_pin.ap_chunk;
  }
  std::vector<int> v;
  if (tune_lookup(kind, ceil_log2_u64(total_queries), ceil_log2_u64(total_db),
                  (int)(n_db * 4096u + n_sets), &v) &&
      v.size() == 1) {
    if (tuned) *tuned = true;
    return v[0];
  }
  return 8192;
}

void ap_chunk_record(uint64_t total_queries, uint64_t total_db, uint32_t n_db, uint32_t n_sets,
                     int chunk, const char* kind) {
  tune_store(kind, ceil_log2_u64(total_queries), ceil_log2_u64(total_db),
             (int)(n_db * 4096u + n_sets), {chunk});
}

}  // namespace bits

using namespace bits;

extern "C" bits_status bits_set_tuning(const bits_tuning* t) {
  if (!t) {
    g_pin = bits_tuning{-1, 0, 0, 0, 0};
    return BITS_OK;
  }
  bool mc_ok = t->mc_shuffles == 0 && t->mc_chunk == 0;
  for (const auto& s : kMcShapes)
    if (t->mc_shuffles == s[0] && t->mc_chunk == s[1]) mc_ok = true;
  bool ap_ok = t->ap_chunk == 0;
  for (int c : kApChunks)
    if (t->ap_chunk == c) ap_ok = true;
  if (t->top_raise < -1 || t->top_raise > kTopRaise ||
      (t->block != 0 && t->block != 256 && t->block != 512) || !mc_ok || !ap_ok) {
    set_error("bits_set_tuning: parameter outside the tuned sets (top_raise -1..2, block "
              "0/256/512, (mc_shuffles, mc_chunk) one of (256,1024) (128,1024) (256,512) "
              "(256,2048) (128,2048) or (0,0), ap_chunk 0/4096/8192/16384/32768)");
    return BITS_EINVAL;
  }
  g_pin = *t;
  return BITS_OK;
}

extern "C" bits_status bits_get_tuning(bits_tuning* t) {
  if (!t) {
    set_error("bits_get_tuning: NULL argument");
    return BITS_EINVAL;
  }
  *t = g_pin;
  return BITS_OK;
}
