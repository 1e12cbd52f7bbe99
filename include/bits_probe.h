/*
 * bits_probe.h -- measurement aid shipped beside the BITS library, in its own
 * shared library (libbits_probe.so, which links against libbits_b300.so for
 * its error reporting: bits_last_error gives the message of a failed call).
 * It is not part of the method (the paper has no counterpart): the
 * benchmark uses it to measure the hardware rate the search kernels are
 * set against.
 */
#ifndef BITS_PROBE_H
#define BITS_PROBE_H

#include "bits.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * bits_probe_random_reads -- the rate at
 * which this GPU serves random 64-byte node reads, the access every search
 * kernel makes once per tree level; on a database much larger than L2 the
 * level-0 reads come from DRAM and this rate bounds the counting kernels.
 * Quads of lanes make uniformly random accesses to d_buf with a 64-byte line
 * fill, four accesses in flight per quad, timed with CUDA events.
 *   d_buf             device buffer, aligned to one access, `bytes` long
 *                     (contents are read, not used); much larger than L2
 *                     (e.g. 4 GiB) for the DRAM rate, well inside it (e.g.
 *                     32 MiB) for the L2 rate.
 *   bytes             a multiple of the access size, at most 2^32 - 1 accesses.
 *   n_reads           accesses to make, 1 .. 2^34 (rounded up to whole rounds
 *                     of the grid).
 *   access_kind       1: one 64-byte node per access (a quad's load);
 *                     2: both 64-byte halves of one random 128-byte line,
 *                     read as two quad loads (a query of the quad descent
 *                     whose start and end searches meet in one interleaved
 *                     node pair); 3: the same line read by one load
 *                     instruction of eight lanes (the octet descent).
 *   h_accesses_per_s  host double receiving the accesses per second.
 * Returns BITS_EINVAL (nothing launched) for a NULL pointer, an access_kind
 * outside 1..3, a misaligned or wrongly sized buffer, or n_reads out of
 * range.  Synchronises `stream`.
 */
bits_status bits_probe_random_reads(const void* d_buf, uint64_t bytes, uint64_t n_reads,
                                    int32_t access_kind, double* h_accesses_per_s,
                                    void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BITS_PROBE_H */
