// CPU oracle for Binary Interval Search (BITS) -- TEST INFRASTRUCTURE ONLY.
//
// This file is the plain, slow, obviously correct statement of what the CUDA
// library computes.  It shares no code, header, table or constant with the
// CUDA library.  Only the test-suite, the package's smoke check and the
// benchmark's CPU-baseline leg load it; the library itself never does.
//
// Conventions (the readings of the paper this oracle follows):
//   * intervals are half-open [start, end) uint32 pairs, so a and b intersect
//     iff b.start < a.end and b.end > a.start (the paper's Sec. "Interval Set
//     Intersection problem" predicate written for half-open intervals);
//   * database intervals must be non-empty (start < end); queries may be
//     empty (start == end) but not inverted (end < start);
//   * self-intersections inside A or inside B are never counted (Sec.
//     "Interval Set Intersection problem");
//   * ICount (Algorithm 1) uses counts, not indices:
//       first = #{ e in B_S : e <  a.end   }   (lower bound of a.end)
//       last  = #{ e in B_E : e <= a.start }   (upper bound of a.start)
//       c     = first - last
//   * Monte-Carlo (Sec. "Monte Carlo Simulations"): A is re-placed, B stays fixed.  Interval i of
//     shuffle s draws Philox4x32-10 with counter (i, s, 0, 0) and key
//     (seed low word, seed high word); u = x1 * 2^32 + x0; its new start is
//     off[c] + floor(u * (len[c] - len_i + 1) / 2^64) inside its own contig c,
//     and it keeps its length.  p = (1 + #{s : T_s >= T_obs}) / (N + 1).
//
// Parity pins for every function live in tests/test_oracle.py.
//
// Build: g++ -O2 -std=c++17 -shared -fPIC -pthread bits_oracle.cpp -o liboracle.so

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// Run f(lo, hi) over [0, n) split into `threads` contiguous pieces.
template <class F>
void parallel_ranges(uint64_t n, int threads, F f) {
  if (threads <= 1 || n < 2) {
    f(uint64_t(0), n);
    return;
  }
  std::vector<std::thread> pool;
  uint64_t per = (n + threads - 1) / threads;
  for (int t = 0; t < threads; ++t) {
    uint64_t lo = uint64_t(t) * per, hi = std::min(n, lo + per);
    if (lo >= hi) break;
    pool.emplace_back([=] { f(lo, hi); });
  }
  for (auto& th : pool) th.join();
}

// Intersection predicate of Sec. "Interval Set Intersection problem", half-open form.
inline bool intersects(uint32_t as, uint32_t ae, uint32_t bs, uint32_t be) {
#ifdef ORACLE_MUTANT_CLOSED
  return bs <= ae && be >= as;  // planted mistake: the closed-interval predicate
#else
  return bs < ae && be > as;
#endif
}

int check_db(const uint32_t* b, uint64_t nb) {
  for (uint64_t j = 0; j < nb; ++j)
    if (!(b[2 * j] < b[2 * j + 1])) return 1;
  return 0;
}

int check_queries(const uint32_t* a, uint64_t na) {
  for (uint64_t i = 0; i < na; ++i)
    if (a[2 * i + 1] < a[2 * i]) return 1;
  return 0;
}

// Algorithm 1: ICount(B_S, B_E, a), both searches as counts.
inline uint32_t icount(const uint32_t* bs, const uint32_t* be, uint64_t nb, uint32_t as,
                       uint32_t ae) {
  uint64_t first = std::lower_bound(bs, bs + nb, ae) - bs;  // #(B_S < a.end)
#ifdef ORACLE_MUTANT_LAST_LOWER
  uint64_t last = std::lower_bound(be, be + nb, as) - be;   // planted: #(B_E < a.start)
#else
  uint64_t last = std::upper_bound(be, be + nb, as) - be;   // #(B_E <= a.start)
#endif
  return uint32_t(first - last);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// 4x32 Philox S-box with multipliers 0xD2511F53 and 0xCD9E8D57 and the Weyl
// key schedule 0x9E3779B9 / 0xBB67AE85 added between rounds.
void philox4x32_10(const uint32_t in_ctr[4], const uint32_t in_key[2], uint32_t out[4]) {
  uint32_t c0 = in_ctr[0], c1 = in_ctr[1], c2 = in_ctr[2], c3 = in_ctr[3];
  uint32_t k0 = in_key[0], k1 = in_key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
#ifdef ORACLE_MUTANT_PHILOX
    uint64_t p0 = uint64_t(0xCD9E8D57u) * c0;  // planted: multipliers swapped
    uint64_t p1 = uint64_t(0xD2511F53u) * c2;
#else
    uint64_t p0 = uint64_t(0xD2511F53u) * c0;
    uint64_t p1 = uint64_t(0xCD9E8D57u) * c2;
#endif
    uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
    uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// floor(u * n / 2^64): the integer map of a uniform 64-bit word onto [0, n).
inline uint64_t scale_u64(uint64_t u, uint64_t n) {
#ifdef ORACLE_MUTANT_SCALE
  return u % n;  // planted: modulo instead of the multiply-high map
#else
  return uint64_t((static_cast<unsigned __int128>(u) * n) >> 64);
#endif
}

// Contig of a genome-wide position: last contig whose offset is <= pos.
inline int64_t contig_of(const uint32_t* coff, uint32_t nc, uint32_t pos) {
  return int64_t(std::upper_bound(coff, coff + nc, pos) - coff) - 1;
}

}  // namespace

extern "C" {

// Brute force over all |A||B| pairs: the definition of Sec. "Interval Set
// Intersection problem" directly. counts (nullable) gets |I(B, a_i)|, total
// gets the size of I(A, B).
int or_count_brute(const uint32_t* a, uint64_t na, const uint32_t* b, uint64_t nb,
                   uint32_t* counts, uint64_t* total) {
  if (check_db(b, nb) || check_queries(a, na)) return 1;
  uint64_t t = 0;
  for (uint64_t i = 0; i < na; ++i) {
    uint32_t as = a[2 * i], ae = a[2 * i + 1];
    uint32_t c = 0;
    for (uint64_t j = 0; j < nb; ++j) c += intersects(as, ae, b[2 * j], b[2 * j + 1]);
    if (counts) counts[i] = c;
    t += c;
  }
  *total = t;
  return 0;
}

// Algorithm 2, first four steps: split B into B_S and B_E and sort each.
int or_build(const uint32_t* b, uint64_t nb, uint32_t* bs, uint32_t* be) {
  if (check_db(b, nb)) return 1;
  for (uint64_t j = 0; j < nb; ++j) {
    bs[j] = b[2 * j];
    be[j] = b[2 * j + 1];
  }
  std::sort(bs, bs + nb);
  std::sort(be, be + nb);
  return 0;
}

// Algorithm 2, counting loop: c = sum over a of ICount(B_S, B_E, a).
int or_count_sorted(const uint32_t* a, uint64_t na, const uint32_t* bs, const uint32_t* be,
                    uint64_t nb, uint32_t* counts, uint64_t* total, int threads) {
  if (check_queries(a, na)) return 1;
  std::vector<uint64_t> part(std::max(1, threads), 0);
  int nt = std::max(1, threads);
  uint64_t per = (na + nt - 1) / nt;
  parallel_ranges(na, nt, [&](uint64_t lo, uint64_t hi) {
    uint64_t t = 0;
    for (uint64_t i = lo; i < hi; ++i) {
      uint32_t c = icount(bs, be, nb, a[2 * i], a[2 * i + 1]);
      if (counts) counts[i] = c;
      t += c;
    }
    part[per ? lo / per : 0] = t;
  });
  uint64_t t = 0;
  for (uint64_t v : part) t += v;
  *total = t;
  return 0;
}

void or_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

uint64_t or_scale_u64(uint64_t u, uint64_t n) { return scale_u64(u, n); }

// New placement of every A interval for shuffle s (Sec. "Monte Carlo Simulations" null model).
// out receives [start, end) pairs.  Returns 1 if an interval is inverted,
// lies outside every contig, or crosses its contig's end.  `set` is the
// index of the query set in a screen of many sets (Sec. "Novel genomic
// relationships"): interval i of set `set` in shuffle s draws the Philox block
// at counter (i, s, set, 0), so every set has its own stream and a single test
// is set 0.
int or_mc_place_set(const uint32_t* a, uint64_t na, const uint32_t* coff, const uint32_t* clen,
                    uint32_t nc, uint64_t seed, uint32_t s, uint32_t set, uint32_t* out) {
  const uint32_t key[2] = {uint32_t(seed), uint32_t(seed >> 32)};
  for (uint64_t i = 0; i < na; ++i) {
    uint32_t as = a[2 * i], ae = a[2 * i + 1];
    if (ae < as) return 1;
    int64_t c = contig_of(coff, nc, as);
    if (c < 0) return 1;
    uint64_t cend = uint64_t(coff[c]) + clen[c];
    if (uint64_t(ae) > cend) return 1;
    uint32_t len = ae - as;
#ifdef ORACLE_MUTANT_SET_WORD
    const uint32_t ctr[4] = {uint32_t(i), s, 0u, set};  // planted: set in word 3
#else
    const uint32_t ctr[4] = {uint32_t(i), s, set, 0u};
#endif
    uint32_t x[4];
    philox4x32_10(ctr, key, x);
#ifdef ORACLE_MUTANT_WORD_ORDER
    uint64_t u = (uint64_t(x[0]) << 32) | x[1];  // planted: words swapped
#else
    uint64_t u = (uint64_t(x[1]) << 32) | x[0];
#endif
    uint64_t range = uint64_t(clen[c]) - len + 1;
    uint64_t start = uint64_t(coff[c]) + scale_u64(u, range);
    out[2 * i] = uint32_t(start);
    out[2 * i + 1] = uint32_t(start + len);
  }
  return 0;
}

// Monte-Carlo significance test (Sec. "Monte Carlo Simulations"): totals[s - s_begin] for each
// shuffle in [s_begin, s_end), the observed total of the unshuffled A, the
// tally k_ge = #{s : T_s >= T_obs} and p = (k_ge + 1) / (N + 1).
int or_mc_set(const uint32_t* a, uint64_t na, const uint32_t* coff, const uint32_t* clen,
              uint32_t nc, const uint32_t* bs, const uint32_t* be, uint64_t nb, uint64_t seed,
              uint32_t s_begin, uint32_t s_end, uint32_t set, uint64_t* totals,
              uint64_t* observed, uint64_t* k_ge, double* pvalue, int threads) {
  if (s_end < s_begin) return 1;
  uint64_t obs = 0;
  if (or_count_sorted(a, na, bs, be, nb, nullptr, &obs, 1)) return 1;
  uint64_t nsh = s_end - s_begin;
  int bad = 0;
  std::vector<int> bad_part(std::max(1, threads), 0);
  uint64_t per = (nsh + std::max(1, threads) - 1) / std::max(1, threads);
  parallel_ranges(nsh, std::max(1, threads), [&](uint64_t lo, uint64_t hi) {
    std::vector<uint32_t> placed(2 * na);
    for (uint64_t k = lo; k < hi; ++k) {
      if (or_mc_place_set(a, na, coff, clen, nc, seed, uint32_t(s_begin + k), set,
                          placed.data())) {
        bad_part[per ? lo / per : 0] = 1;
        return;
      }
      uint64_t t = 0;
      for (uint64_t i = 0; i < na; ++i) t += icount(bs, be, nb, placed[2 * i], placed[2 * i + 1]);
      totals[k] = t;
    }
  });
  for (int v : bad_part) bad |= v;
  if (bad) return 1;
  uint64_t k = 0;
#ifdef ORACLE_MUTANT_TALLY
  for (uint64_t j = 0; j < nsh; ++j) k += totals[j] > obs;  // planted: strict tally
#else
  for (uint64_t j = 0; j < nsh; ++j) k += totals[j] >= obs;
#endif
  *observed = obs;
  *k_ge = k;
  *pvalue = double(k + 1) / double(nsh + 1);
  return 0;
}

int or_mc_place(const uint32_t* a, uint64_t na, const uint32_t* coff, const uint32_t* clen,
                uint32_t nc, uint64_t seed, uint32_t s, uint32_t* out) {
  return or_mc_place_set(a, na, coff, clen, nc, seed, s, 0u, out);
}

int or_mc(const uint32_t* a, uint64_t na, const uint32_t* coff, const uint32_t* clen,
          uint32_t nc, const uint32_t* bs, const uint32_t* be, uint64_t nb, uint64_t seed,
          uint32_t s_begin, uint32_t s_end, uint64_t* totals, uint64_t* observed,
          uint64_t* k_ge, double* pvalue, int threads) {
  return or_mc_set(a, na, coff, clen, nc, bs, be, nb, seed, s_begin, s_end, 0u, totals, observed,
                   k_ge, pvalue, threads);
}

// Summary of one Monte-Carlo test (Sec. "Monte Carlo Simulations", Sec. "Novel
// genomic relationships" and Fig. 3):
//   ints[0] observed total        ints[1] k_ge = #{s : T_s >= observed}
//   ints[2] k_le = #{s : T_s <= observed}
//   ints[3], ints[4] the two middle totals of the sorted T, at ranks
//           floor((N - 1) / 2) and floor(N / 2) (equal for odd N); the median
//           is their mean
//   dbl[0] enrichment p = (k_ge + 1) / (N + 1)
//   dbl[1] depletion p  = (k_le + 1) / (N + 1)
//   dbl[2] Fig. 3's enrichment score log2(observed / median), evaluated as
//          log2(double(2 * observed) / double(lo + hi)) (IEEE: 0 / 0 is NaN,
//          x / 0 is +inf, log2(0) is -inf).
// N = 0 gives zero middles and p = 1.  Returns 1 on 64-bit overflow of
// 2 * observed or lo + hi.
int or_mc_summary(const uint64_t* totals, uint64_t n, uint64_t observed, uint64_t* ints,
                  double* dbl) {
  std::vector<uint64_t> t(totals, totals + n);
  std::sort(t.begin(), t.end());
  uint64_t kge = 0, kle = 0;
  for (uint64_t v : t) {
    kge += v >= observed;
#ifdef ORACLE_MUTANT_DEPLETE
    kle += v < observed;  // planted: strict depletion tally
#else
    kle += v <= observed;
#endif
  }
#ifdef ORACLE_MUTANT_MEDIAN
  const uint64_t lo = n ? t[n / 2] : 0, hi = n ? t[n / 2] : 0;  // planted: upper middle twice
#else
  const uint64_t lo = n ? t[(n - 1) / 2] : 0, hi = n ? t[n / 2] : 0;
#endif
  if (observed > UINT64_MAX / 2 || lo > UINT64_MAX - hi) return 1;
  ints[0] = observed;
  ints[1] = kge;
  ints[2] = kle;
  ints[3] = lo;
  ints[4] = hi;
  dbl[0] = double(kge + 1) / double(n + 1);
  dbl[1] = double(kle + 1) / double(n + 1);
  dbl[2] = std::log2(double(2 * observed) / double(lo + hi));
  return 0;
}

// Enumeration problem (Sec. "Interval Set Intersection problem": report every
// intersecting pair), by the definition: for each query i in order, every
// database interval j in index order with b_j meeting a_i.  offsets[i] is the
// first pair of query i and offsets[na] the number of pairs; pairs (if not
// NULL) receives (i, j) words.
int or_enumerate_brute(const uint32_t* a, uint64_t na, const uint32_t* b, uint64_t nb,
                       uint64_t* offsets, uint32_t* pairs) {
  if (check_db(b, nb) || check_queries(a, na)) return 1;
  uint64_t k = 0;
  for (uint64_t i = 0; i < na; ++i) {
    offsets[i] = k;
    for (uint64_t j = 0; j < nb; ++j)
      if (intersects(a[2 * i], a[2 * i + 1], b[2 * j], b[2 * j + 1])) {
        if (pairs) {
          pairs[2 * k] = uint32_t(i);
          pairs[2 * k + 1] = uint32_t(j);
        }
        ++k;
      }
  }
  offsets[na] = k;
  return 0;
}

// Enumeration the way Sec. "BITS Algorithm" sets it up: B sorted by start (ties in index
// order) with each entry's end and index beside it; ICount gives the number
// c of intervals meeting a, and since every one of them starts before
// a.end, scanning the entries left of first = #(B_S < a.end) from right to
// left and keeping those with end > a.start finds all of them; the scan
// stops at the c-th (|I| as the termination condition).  Pairs of a query
// come in scan order: descending start, then descending index.
int or_enumerate_scan(const uint32_t* a, uint64_t na, const uint32_t* b, uint64_t nb,
                      uint64_t* offsets, uint32_t* pairs) {
  if (check_db(b, nb) || check_queries(a, na)) return 1;
  std::vector<uint32_t> bs(nb), be(nb), idx(nb);
  for (uint64_t j = 0; j < nb; ++j) {
    bs[j] = b[2 * j];
    be[j] = b[2 * j + 1];
    idx[j] = uint32_t(j);
  }
  std::sort(bs.begin(), bs.end());
  std::sort(be.begin(), be.end());
  std::stable_sort(idx.begin(), idx.end(),
                   [&](uint32_t x, uint32_t y) { return b[2 * x] < b[2 * y]; });
  uint64_t k = 0;
  for (uint64_t i = 0; i < na; ++i) {
    offsets[i] = k;
    const uint32_t as = a[2 * i], ae = a[2 * i + 1];
    const uint32_t c = icount(bs.data(), be.data(), nb, as, ae);
    const uint64_t first = std::lower_bound(bs.begin(), bs.end(), ae) - bs.begin();
    uint32_t found = 0;
    for (uint64_t p = first; p > 0 && found < c; --p) {
      const uint32_t j = idx[p - 1];
#ifdef ORACLE_MUTANT_ENUM_END
      if (b[2 * j + 1] >= as) {  // planted: touching ends counted as hits
#else
      if (b[2 * j + 1] > as) {
#endif
        if (pairs) {
          pairs[2 * (k + found)] = uint32_t(i);
          pairs[2 * (k + found) + 1] = j;
        }
        ++found;
      }
    }
    k += c;
  }
  offsets[na] = k;
  return 0;
}

// The predicate of Sec. "Interval Set Intersection problem" exactly as
// printed, for closed intervals [start, end]: a and b intersect iff a.start <=
// b.end and a.end >= b.start.  Brute force.
int or_count_brute_closed(const uint32_t* a, uint64_t na, const uint32_t* b, uint64_t nb,
                          uint32_t* counts, uint64_t* total) {
  for (uint64_t j = 0; j < nb; ++j)
    if (b[2 * j + 1] < b[2 * j]) return 1;
  if (check_queries(a, na)) return 1;
  uint64_t t = 0;
  for (uint64_t i = 0; i < na; ++i) {
    uint32_t c = 0;
    for (uint64_t j = 0; j < nb; ++j)
#ifdef ORACLE_MUTANT_BRUTE_CLOSED
      c += (a[2 * i] < b[2 * j + 1] && a[2 * i + 1] > b[2 * j]) ? 1u : 0u;
#else
      c += (a[2 * i] <= b[2 * j + 1] && a[2 * i + 1] >= b[2 * j]) ? 1u : 0u;
#endif
    if (counts) counts[i] = c;
    t += c;
  }
  *total = t;
  return 0;
}

// Projection of chromosome-local intervals onto one line (Sec. "BITS
// Algorithm" (projection)): interval i on contig chrom[i] becomes [off[chrom]
// + start, off[chrom] + end), with one added to the end for closed input,
// since [s, e] on the integers is [s, e + 1).  With no contig table (nc == 0)
// every interval is on one contig at offset 0 that spans the whole 32-bit
// line.  An interval that cannot be projected (contig id out of range, start >
// end, end past its contig, or an end that does not fit in 32 bits) is written
// as the inverted pair (2^32 - 1, 0), which every counting call rejects; the
// return value is the number of such intervals.
uint64_t or_project(const uint32_t* chrom, const uint32_t* start, const uint32_t* end, uint64_t n,
                    const uint32_t* coff, const uint32_t* clen, uint32_t nc, int closed,
                    uint32_t* out) {
  uint64_t bad = 0;
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t off = 0, len = 0xFFFFFFFFull;
    bool ok = true;
    if (nc) {
      const uint32_t c = chrom[i];
      ok = c < nc;
      if (ok) {
        off = coff[c];
        len = clen[c];
      }
    }
#ifdef ORACLE_MUTANT_PROJECT_CLOSED
    const uint64_t e = uint64_t(end[i]);
#else
    const uint64_t e = uint64_t(end[i]) + (closed ? 1u : 0u);
#endif
#ifdef ORACLE_MUTANT_PROJECT_OFFSET
    if (nc && ok) off = coff[0];
#endif
    ok = ok && start[i] <= end[i] && e <= len && off + e <= 0xFFFFFFFFull;
    if (ok) {
      out[2 * i] = uint32_t(off + start[i]);
      out[2 * i + 1] = uint32_t(off + e);
    } else {
      out[2 * i] = 0xFFFFFFFFu;
      out[2 * i + 1] = 0u;
      ++bad;
    }
  }
  return bad;
}

}  // extern "C"
