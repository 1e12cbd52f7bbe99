/*
 * bits.h -- C ABI of the B300 (sm_103a) Binary Interval Search library.
 *
 * Binary Interval Search (BITS; Layer, Skadron, Robins, Hall and Quinlan,
 * Bioinformatics 2012) counts interval intersections by exclusion: for a
 * query a and a database B split into independently sorted start and end
 * arrays B_S and B_E, the number of database intervals meeting a is
 *     ICount(a) = #(B_S < a.end) - #(B_E <= a.start)           (Algorithm 1)
 * which equals |B| minus the intervals wholly right of a, minus those wholly
 * left of a (Sec. "BITS Algorithm", the sets L and R).  The counting problem
 * sums ICount over A (Algorithm 2); the Monte-Carlo significance test (Sec.
 * "Monte Carlo Simulations") recounts after re-placing A at random many
 * times.  Passages are cited by the title of their subsection.
 *
 * Conventions shared by every call:
 *   - Intervals are half-open [start, end) pairs of uint32 on one genome-wide
 *     coordinate line (contigs already projected by adding their offsets, as
 *     the projection paragraph of Sec. "BITS Algorithm" describes).  An
 *     interval set is an array of structures: element i is the two
 *     consecutive words (start_i, end_i), 8 bytes per interval.
 *     a and b intersect iff b.start < a.end and b.end > a.start.
 *   - Database intervals must be non-empty (start < end).  Queries may be
 *     empty (start == end) and then count the database intervals with
 *     start < x < end; queries with end < start are invalid.
 *   - Pointers named d_* are device pointers on the current CUDA device, h_*
 *     are host pointers.  The caller owns every pointer it passes; the library
 *     never frees them.  A bits_db owns its own device memory until bits_free.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered; a call that returns host values
 *     synchronises that stream first.
 *   - Every call returns a bits_status; on failure bits_last_error() gives a
 *     message (thread-local).  No call falls back to host computation.
 *   - Device memory comes from a stream-ordered pool the library creates
 *     per device at first use: a database's own storage (one block, freed
 *     by bits_free) and every temporary (sort buffers, merge-path keys,
 *     enumeration counts, staging of pageable host buffers).  Up to 4 GiB
 *     of freed memory stays reserved in it for reuse by later calls and
 *     databases, for the life of the process.
 */
#ifndef BITS_H
#define BITS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bits_db bits_db;

typedef enum bits_status {
  BITS_OK = 0,
  BITS_EINVAL = 1,     /* bad argument, or an invalid interval was seen          */
  BITS_ENOMEM = 2,     /* device allocation failed                               */
  BITS_ECUDA = 3,      /* CUDA runtime error (message in bits_last_error)        */
  BITS_EOVERFLOW = 4,  /* a size beyond the supported range                      */
  BITS_ETIMEOUT = 5,   /* a bounded device-side wait gave up; results invalid    */
  BITS_ENOTIMPL = 6,   /* method not built into this database                    */
  BITS_EINTERNAL = 7   /* a device-side consistency check failed (a library bug,  */
                       /* e.g. a sort scatter index out of range); results invalid */
} bits_status;

typedef enum bits_method {
  BITS_METHOD_AUTO = 0,      /* autotuner picks among the built methods            */
  BITS_METHOD_SEARCH = 1,    /* shared-memory top + quad-cooperative 16-ary tree   */
  BITS_METHOD_RMI = 2,       /* learned index: predict, bounded search, verify     */
  BITS_METHOD_MERGEPATH = 3  /* sort the queries, co-rank them by merge path       */
} bits_method;

/* Build options; pass NULL for the defaults (every field 0). */
typedef struct bits_opts {
  int32_t method;          /* bits_method the database uses by default           */
  int32_t rmi_leaves_log2; /* 0: no learned index; else 2^k linear leaves per     */
                           /* sorted array, k in [1, 22]                          */
  int32_t top_tree_log2;   /* 0: default 12; the top level of each array's        */
                           /* 16-ary search tree kept in shared memory holds at   */
                           /* most 2^k - 1 keys, k in [2, 14]                     */
  int32_t flags;           /* BITS_FLAG_* bits; 0 for none                        */
} bits_opts;

/* Keep the database intervals in start order as (end, index) pairs, 8 more
 * bytes per interval, so that bits_enumerate_pairs can report pairs. */
#define BITS_FLAG_ENUMERATE 1

/*
 * bits_build_db -- Algorithm 2's set-up: B_S <- starts, B_E <- ends, sort both.
 *   d_b   device, n intervals as (start, end) uint32 pairs; read only.
 *   n     number of database intervals, 0 <= n < 2^30 (else BITS_EOVERFLOW).
 *   out   receives the new database handle (owns B_S, B_E, search tree and
 *         the optional learned index).
 * Device memory per database: about 16.5 bytes per interval (B_S and B_E,
 * their levels stored once more with node i of both arrays in one 128-byte
 * line for the searches, and the upper levels), plus 64 bytes per pair of
 * learned-index leaves and 8 bytes per interval with BITS_FLAG_ENUMERATE.
 * Sorting is the library's own LSD radix sort.  The call synchronises the
 * stream once (it reads the validation flag): BITS_EINVAL if any interval has
 * end <= start, in which case *out is left NULL.
 */
bits_status bits_build_db(const uint32_t* d_b, uint64_t n, const bits_opts* opts, void* stream,
                          bits_db** out);

/*
 * bits_count -- Algorithm 2's counting loop over Algorithm 1.
 *   d_a       device, n queries as (start, end) uint32 pairs; read only.
 *   n         number of queries, n < 2^32.
 *   d_counts  device uint32[n] receiving ICount(a_i), or NULL to skip.
 *   d_total   device uint64[1] receiving the sum over all queries.
 * Asynchronous.  Inverted queries (end < start) count 0 and set the
 * database's device error word; bits_check reports it as BITS_EINVAL.
 */
bits_status bits_count(const bits_db* db, const uint32_t* d_a, uint64_t n, uint32_t* d_counts,
                       uint64_t* d_total, void* stream);

/* Same as bits_count with an explicit method (for side-by-side comparison). */
bits_status bits_count_method(const bits_db* db, int32_t method, const uint32_t* d_a,
                              uint64_t n, uint32_t* d_counts, uint64_t* d_total, void* stream);

/*
 * bits_count_host -- bits_count_method on host buffers: the queries come
 * from host memory and the counts and the total go back to it within the
 * one call (Algorithm 2 over Algorithm 1, as bits_count).
 *   method    a bits_method; AUTO takes the choice the autotuner made for
 *             this size class (plain search until one has been tuned).
 *   h_a       host, n queries as (start, end) uint32 pairs, 8-byte aligned.
 *   n         number of queries, n < 2^32.
 *   h_counts  host uint32[n] receiving ICount(a_i), 4-byte aligned, or NULL.
 *   h_total   host uint64 receiving the sum over all queries, 8-byte aligned.
 * Page-locked buffers (cudaHostAlloc, cudaMallocHost, cudaHostRegister; the
 * whole range inside one such allocation) are read and written in place by
 * the search kernel over the bus, so the transfers overlap the searches and
 * nothing is staged.  Pageable buffers are staged through stream-ordered
 * device memory with cudaMemcpyAsync; merge path always stages.  The total
 * is added up in a stream-ordered device word of the call's own and copied
 * to h_total; that memory comes from the library's pool.  Stream-ordered
 * like every call: with page-locked buffers it returns at once and the
 * results are in place when `stream` has been synchronised; a pageable
 * h_total or h_counts makes the call wait for its copy, as cudaMemcpyAsync
 * does.  Inverted queries count
 * 0 and set the database's device error word (bits_check).  BITS_EINVAL if a
 * buffer is device memory or the database belongs to another device than
 * the current one.
 */
bits_status bits_count_host(const bits_db* db, int32_t method, const uint32_t* h_a, uint64_t n,
                            uint32_t* h_counts, uint64_t* h_total, void* stream);

/*
 * Enumeration problem (Sec. "Interval Set Intersection problem": report every
 * intersecting pair), in two stream-ordered steps so that the caller can size
 * the output in between.
 *
 * bits_enumerate_offsets -- d_offsets (device uint64[n + 1]) receives the
 * exclusive prefix sum of ICount over the queries: query i's pairs occupy
 * [d_offsets[i], d_offsets[i + 1]) and d_offsets[n] is the number of pairs.
 * Asynchronous; inverted queries count 0 and set the device error word.
 *
 * bits_enumerate_pairs -- writes the pairs, as (query index, database
 * interval index) uint32 pairs in d_pairs (device, 8-byte aligned,
 * d_offsets[n] pairs), given the offsets of the same queries and database.
 * Needs a database built with BITS_FLAG_ENUMERATE (else BITS_ENOTIMPL).  As
 * Sec. "BITS Algorithm" suggests, ICount ends the scan: the database
 * intervals in start order left of first = #(B_S < a.end) are walked right to
 * left and those with end > a.start kept until the count is reached, so a
 * query's pairs come in descending start order (equal starts: descending
 * index).  A query
 * under a long interval that contains many others scans past them (the
 * paper's containment case).  Asynchronous; offsets that do not match the
 * queries set the device error word (bits_check: BITS_EINVAL).
 */
bits_status bits_enumerate_offsets(const bits_db* db, const uint32_t* d_a, uint64_t n,
                                   uint64_t* d_offsets, void* stream);
bits_status bits_enumerate_pairs(const bits_db* db, const uint32_t* d_a, uint64_t n,
                                 const uint64_t* d_offsets, uint32_t* d_pairs, void* stream);

/*
 * bits_mc -- Monte-Carlo significance test of Sec. "Monte Carlo
 * Simulations".  Each shuffle s in [shuffle_begin, shuffle_end) re-places
 * every query interval uniformly inside its own contig with its length kept,
 * and recounts it against the fixed database.  Interval i of shuffle s draws Philox4x32-10 with counter
 * (i, s, 0, 0) and key (seed & 0xffffffff, seed >> 32); with u = x1*2^32 + x0
 * its new start is off[c] + floor(u * (len[c] - len_i + 1) / 2^64).
 *   d_contig_off, d_contig_len  device uint32[n_contigs], the contig table on
 *                               the same coordinate line (offsets ascending).
 *   d_totals    device uint64[shuffle_end - shuffle_begin], per-shuffle totals.
 *   h_observed  host, total of the unshuffled queries (nullable).
 *   h_k_ge      host, #{s : total_s >= observed} (nullable).
 *   h_pvalue    host, (k_ge + 1) / (N + 1) in IEEE double (nullable).
 * method: BITS_METHOD_SEARCH or BITS_METHOD_RMI (AUTO: SEARCH).  Synchronises the
 * stream.  BITS_EINVAL if a query is inverted, lies before the first contig or
 * crosses its contig's end.  Work of one call runs as one persistent launch,
 * replayed from a cached CUDA graph when the same arguments repeat.
 */
bits_status bits_mc(const bits_db* db, int32_t method, const uint32_t* d_a, uint64_t n,
                    const uint32_t* d_contig_off, const uint32_t* d_contig_len,
                    uint32_t n_contigs, uint64_t seed, uint32_t shuffle_begin,
                    uint32_t shuffle_end, uint64_t* d_totals, uint64_t* h_observed,
                    uint64_t* h_k_ge, double* h_pvalue, void* stream);

/*
 * Summary of one Monte-Carlo test (64 bytes).  With N shuffled totals T_s:
 *   k_ge, k_le    #{s : T_s >= observed}, #{s : T_s <= observed}
 *   median_lo/hi  the sorted totals at ranks floor((N-1)/2) and floor(N/2)
 *                 (equal for odd N); the median is their mean
 *   p_enrich      (k_ge + 1) / (N + 1), one IEEE double division
 *   p_deplete     (k_le + 1) / (N + 1)
 *   log2_enrichment  Fig. 3's enrichment score log2(observed / median),
 *                 evaluated as log2(double(2 * observed) / double(lo + hi))
 *                 with IEEE specials (0/0 gives NaN, x/0 +inf, log2(0)
 *                 -inf); NaN as well if 2 * observed or lo + hi overflows.
 */
typedef struct bits_mc_stat {
  uint64_t observed;
  uint64_t k_ge;
  uint64_t k_le;
  uint64_t median_lo;
  uint64_t median_hi;
  double p_enrich;
  double p_deplete;
  double log2_enrichment;
} bits_mc_stat;

/*
 * bits_mc_summary -- bits_mc_stat of n_tests Monte-Carlo tests at once (the
 * tally of Sec. "Monte Carlo Simulations" in both directions and the Fig. 3
 * score).
 *   d_totals    device uint64[n_tests][n_shuffles], row t = test t's totals.
 *   d_observed  device uint64[n_tests].
 *   d_stats     device bits_mc_stat[n_tests], 8-byte aligned.
 * One CTA per test; asynchronous.  The score's log2 is CUDA's (at most 1 ulp
 * from the exact value); every other field is exact.
 */
bits_status bits_mc_summary(const uint64_t* d_totals, uint32_t n_shuffles, uint32_t n_tests,
                            const uint64_t* d_observed, bits_mc_stat* d_stats, void* stream);

/*
 * bits_mc_matrix -- the Monte-Carlo screen of Sec. "Novel genomic
 * relationships": a significance test (Sec. "Monte Carlo Simulations") for
 * every pair of query set A_i and database B_j.
 *   dbs, n_db, d_as, n_as, n_sets   as bits_count_matrix.
 *   d_contig_off, d_contig_len, n_contigs, seed, shuffle_begin, shuffle_end
 *                as bits_mc; one contig table for every set (n_contigs <= 4096).
 *   d_observed   device uint64[n_sets][n_db]: total(A_i, B_j) (bits_count_matrix).
 *   d_totals     device uint64[n_sets][n_db][N], N = shuffle_end - shuffle_begin:
 *                the total of shuffle s for pair (i, j) at [i][j][s - begin].
 *   d_stats      device bits_mc_stat[n_sets][n_db], or NULL to skip.
 * Interval k of set i in shuffle s draws Philox4x32-10 at counter
 * (k, s, i, 0), so set i is re-placed the same way against every database and
 * set 0 reproduces bits_mc.  Asynchronous: invalid query intervals set the
 * error word of each database they were counted against (bits_check).  The
 * shuffle work of all pairs is one persistent launch, replayed from a cached
 * CUDA graph when the same arguments repeat.  Work units above 2^32 (about
 * 1.1e15 placements) give BITS_EOVERFLOW: split the shuffle range.  When the
 * sets are large against many databases (searching every placement in every
 * database would cost at least twice as much) and every query interval is
 * non-empty and inside its contig, the call instead builds the sets, then
 * each shuffle's placed sets, as databases of their own and counts every
 * pair from its smaller side (as bits_count_matrix_db); the same draws give
 * the same totals, and the call then returns only after the device has
 * finished its work (it frees the sets' databases, as bits_free does).
 */
bits_status bits_mc_matrix(const bits_db* const* dbs, uint32_t n_db, const uint32_t* const* d_as,
                           const uint64_t* n_as, uint32_t n_sets, const uint32_t* d_contig_off,
                           const uint32_t* d_contig_len, uint32_t n_contigs, uint64_t seed,
                           uint32_t shuffle_begin, uint32_t shuffle_end, uint64_t* d_observed,
                           uint64_t* d_totals, bits_mc_stat* d_stats, void* stream);

/*
 * bits_count_matrix -- all-pairs screen of Sec. "Novel genomic relationships":
 * M[i][j] = total(A_i, B_j).
 *   dbs      host array of n_db database handles (all on this device).
 *   d_as     host array of n_sets device pointers to query sets.
 *   n_as     host array of n_sets query-set sizes.
 *   d_matrix device uint64[n_sets][n_db], row-major.
 * One persistent launch over (query chunk, database) work units ordered by
 * cost; asynchronous.
 */
bits_status bits_count_matrix(const bits_db* const* dbs, uint32_t n_db,
                              const uint32_t* const* d_as, const uint64_t* n_as, uint32_t n_sets,
                              uint64_t* d_matrix, void* stream);

/*
 * bits_count_matrix_db -- the same matrix when the query sets are databases
 * too (the paper's screen compares every track with every other, so each is
 * both): M[i][j] = total(A_i, B_j) from the sorted arrays alone.  Algorithm
 * 2's sum of ICount over A splits into one rank sum per array,
 *     total(A, B) = sum_{x in A_E} #(B_S < x) - sum_{x in A_S} #(B_E <= x),
 * and counting the same pairs from B's side gives the mirror image, so each
 * pair is counted from its smaller side's keys: searched in its larger
 * side's tree (min(|A_i|, |B_j|) searches instead of |A_i|, keys in order),
 * or, when the two sides are within a factor 8 in size, read off a merge of
 * the sorted arrays.
 *   a_dbs, n_a  host array of the query sets' database handles.
 *   b_dbs, n_b  host array of the databases' handles (all on this device).
 *   d_matrix    device uint64[n_a][n_b], row-major.
 * Gives the same matrix as bits_count_matrix on the sets' intervals (database
 * intervals are never empty or inverted, so no query is left out).  One
 * persistent launch over (key chunk, tree) work units, largest tree first,
 * and two over the merge tiles, replayed from a cached CUDA graph;
 * asynchronous.
 */
bits_status bits_count_matrix_db(const bits_db* const* a_dbs, uint32_t n_a,
                                 const bits_db* const* b_dbs, uint32_t n_b, uint64_t* d_matrix,
                                 void* stream);

/*
 * bits_project -- the mapping of Sec. "BITS Algorithm" (projection) that
 * places every chromosome after the previous ones on one genome-wide line, and
 * the conversion of closed intervals (Sec. "Interval Set Intersection problem"
 * states its predicate for closed [start, end]) to the half-open form every
 * other call takes: [s, e] on the integers is [s, e + 1).  Interval i on
 * chromosome c = d_contig[i] becomes [off[c] + start_i, off[c] + end_i), plus
 * one on the end when closed.
 *   d_contig      device uint32[n], chromosome ids; ignored (may be NULL) when
 *                 n_contigs == 0, which means one line at offset 0 with
 *                 length 2^32 - 1.
 *   d_start, d_end  device uint32[n], coordinates local to the chromosome.
 *   d_contig_off, d_contig_len  device uint32[n_contigs].
 *   closed        0: input is half-open [start, end); 1: closed [start, end].
 *   d_out         device, n (start, end) uint32 pairs, 8-byte aligned; must
 *                 not overlap the inputs.
 *   d_n_rejected  device uint64[1] or NULL: set to the number of rejected rows.
 * A row is rejected when its chromosome id is >= n_contigs, start > end, its
 * half-open end passes the chromosome's length, or the projected end passes
 * 2^32 - 1.  It is written as the inverted pair (2^32 - 1, 0), which
 * bits_build_db and every counting call reject (BITS_EINVAL), so a rejected
 * row cannot be counted by mistake.  Asynchronous; one kernel launch.
 */
bits_status bits_project(const uint32_t* d_contig, const uint32_t* d_start, const uint32_t* d_end,
                         uint64_t n, const uint32_t* d_contig_off, const uint32_t* d_contig_len,
                         uint32_t n_contigs, int32_t closed, uint32_t* d_out,
                         uint64_t* d_n_rejected, void* stream);

/*
 * bits_sort_intervals_noalloc -- the paper has no counterpart; this is a
 * service for callers that cannot allocate device memory: code whose device
 * memory is entirely owned by another allocator (a framework's caching pool
 * that reserves the GPU up front), serving loops that fix their memory plan
 * at start-up, and callers that cannot afford cudaMalloc's implicit
 * synchronisation.  It sorts the start words and the end words of n
 * intervals into d_bs and d_be -- the same arrays bits_build_db builds -- and
 * allocates nothing: its scratch (about 2.4 MB) is a fixed array inside the
 * library that every GPU loading the library holds until the process exits.
 *   d_b    device, n (start, end) uint32 pairs, 8-byte aligned; read only.
 *   n      0 <= n <= BITS_NOALLOC_MAX_INTERVALS, else BITS_EOVERFLOW.
 *   d_bs   device uint32[n], receives the sorted starts (caller-owned).
 *   d_be   device uint32[n], receives the sorted ends (caller-owned).
 * The first call on a device also looks up the scratch array's device
 * address (cudaGetSymbolAddress).
 * All calls on a device share the one scratch array: calls that overlap on
 * the GPU (other streams, other host threads) race and must be serialised
 * by the caller.  The call synchronises `stream` (it reads the sort's digit
 * histograms and its error word back).  BITS_EINVAL if an interval has
 * end <= start; the error word is cleared at the start of every call, so a
 * later valid call succeeds.  BITS_EINTERNAL if the sort's own consistency
 * check fails (a library bug).
 */
#define BITS_NOALLOC_MAX_INTERVALS 262144u
bits_status bits_sort_intervals_noalloc(const uint32_t* d_b, uint64_t n, uint32_t* d_bs,
                                        uint32_t* d_be, void* stream);

/*
 * Launch parameters (the paper has none of these; none changes a result).
 * Every call lays out its work with parameters it takes, per field, from
 * the values pinned on the calling host thread by bits_set_tuning, else from
 * the autotuner's record for its size class, else from the defaults.  A
 * size class is (device, ceil log2 of the queries, ceil log2 of the
 * database, learned index built or not, per-query counts wanted or not, the
 * method named).  The first bits_count / bits_count_method call of a class
 * that nothing pins times the candidates on the caller's own inputs with
 * CUDA events (batches of back-to-back calls, three alternating rounds) and
 * records the fastest of each method (used by calls that name their
 * method) and, for BITS_METHOD_AUTO, the fastest plain search unless another
 * method is at least 5 % faster (with no record -- parameters pinned, or
 * under stream capture -- AUTO takes the plain search); bits_mc and
 * bits_count_matrix time their own candidates the same way on their first
 * call of a class.  Nothing is timed under stream capture.  When the
 * environment variable BITS_AUTOTUNE_CACHE names a file, records are read
 * from it at first use and appended to it as they are made, one line each:
 *     <device> <kind> <log2 queries> <log2 database> <flags> <values...>
 * with kind "count" (values: method, top_raise, block), "mc" (mc_shuffles,
 * mc_chunk, top_raise) or "allpairs" (ap_chunk).
 */
typedef struct bits_tuning {
  int32_t top_raise;    /* plain search in bits_count and bits_mc: levels above the
                           database's default shared-memory top level to keep in shared
                           memory instead (0, 1 or 2: a 16x, 256x smaller top, one or two
                           more tree levels read from memory); -1: tuned */
  int32_t block;        /* bits_count search kernels: threads per CTA, 256 or 512; 0: tuned */
  int32_t mc_shuffles;  /* bits_mc: shuffles per work unit (threads per CTA), and */
  int32_t mc_chunk;     /* intervals per work unit, one of the pairs (256, 1024),
                           (128, 1024), (256, 512), (256, 2048), (128, 2048); (0, 0): tuned */
  int32_t ap_chunk;     /* bits_count_matrix: queries per work unit, 4096, 8192, 16384 or
                           32768; 0: tuned */
} bits_tuning;

/* Pin launch parameters for later calls on this host thread (NULL: unpin
 * everything).  BITS_EINVAL, and nothing changes, if a field is outside the
 * sets listed above. */
bits_status bits_set_tuning(const bits_tuning* t);

/* The parameters pinned on this host thread (fields at -1 / 0 are tuned). */
bits_status bits_get_tuning(bits_tuning* t);

/*
 * bits_selftest_wait -- diagnostic of the bounded device-side waits (not in
 * the paper).  Every spin-wait of the library (the radix sort's look-back)
 * gives up after a fixed number of iterations, records a timeout and
 * returns, so a lost peer cannot hang the GPU.  This call runs the same kind
 * of wait on a device word that nothing sets, with spin_limit iterations
 * (1 .. 2^23, each sleeping about 64 ns): it returns BITS_ETIMEOUT, and the
 * context stays usable.  Synchronises `stream`.
 */
bits_status bits_selftest_wait(uint32_t spin_limit, void* stream);

/* Read-only views of the database (sorted starts, sorted ends, size). */
bits_status bits_db_info(const bits_db* db, const uint32_t** d_bs, const uint32_t** d_be,
                         uint64_t* n, int32_t* has_rmi);

/*
 * bits_db_rmi -- the learned index of one sorted array (which = 0: starts,
 * 1: ends), for inspection.  The leaf table is device memory owned by the
 * database: n_leaves records of 32 bytes, each
 *     uint32 base_key, uint32 lo, float slope, float icpt,
 *     int32 err_lo, int32 err_hi, uint32 hi, uint32 reserved
 * (leaf l owns ranks [lo, hi) of the sorted array and predicts the rank of a
 * key k as lo + round(slope * (k - base_key) + icpt), clamped, with the true
 * rank inside [prediction + err_lo, prediction + err_hi]).  The root maps k
 * to leaf floor(root_slope * k + root_icpt), clamped to [0, n_leaves).
 * bits_build_db fits both stages on the device as least-squares lines of
 * rank against key, from exact integer sums over the sorted array, and then
 * measures every leaf's error bounds with the search's own prediction, so
 * counts through the index equal the plain search's whatever the fit.
 * The learned index is not in the paper; it narrows each BSearch of
 * Algorithm 1 before an exact search finishes it.  BITS_ENOTIMPL without one.
 */
bits_status bits_db_rmi(const bits_db* db, int32_t which, const void** d_leaves,
                        uint32_t* n_leaves, float* root_slope, float* root_icpt);

/* Synchronise `stream`, then return and clear the database's device error word. */
bits_status bits_check(const bits_db* db, void* stream);

/* Release a database (NULL-safe): waits for all work on its device, then
 * returns its memory to the library's pool. */
void bits_free(bits_db* db);

/* Message of the last failing call on this host thread ("" if none). */
const char* bits_last_error(void);

/* Number of kernels this library has launched in this process. */
uint64_t bits_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* BITS_H */
