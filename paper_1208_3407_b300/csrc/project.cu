// Projection onto one coordinate line (Sec. "BITS Algorithm" (projection)) and closed-to-half-open
// conversion (Sec. "Interval Set Intersection problem" states its predicate for closed intervals).
//
// Interval i on chromosome c = chrom[i] becomes [off[c] + start, off[c] + end)
// (end + 1 for closed input, since [s, e] on the integers is [s, e + 1)).
// The work is a pure stream: 12 bytes read (chrom, start, end) and 8 bytes
// written per interval, so the kernel is HBM-bound.  Each thread maps four
// consecutive intervals with 16-byte loads and stores when every pointer is
// 16-byte aligned; a scalar loop covers the ragged tail and unaligned calls.
// The chromosome table is read through the read-only cache (it is small and
// every warp reuses it).  A row that cannot be mapped is written as the
// inverted pair (2^32 - 1, 0), which every counting call rejects, and counted
// into an optional device word with one atomic per warp.
#include "common.cuh"
#include "project.cuh"

namespace bits {
namespace {

constexpr int kProjBlock = 256;

struct ProjArgs {
  const uint32_t* chrom;
  const uint32_t* start;
  const uint32_t* end;
  uint64_t n;
  const uint32_t* off;
  const uint32_t* len;
  uint32_t n_contigs;
  uint32_t closed;
  uint2* out;
  unsigned long long* n_rejected;
};

__device__ __forceinline__ uint2 project_one(const ProjArgs& P, uint32_t c, uint32_t s, uint32_t e,
                                             uint32_t& bad) {
  uint64_t o = 0, l = kU32Max;
  bool ok = true;
  if (P.n_contigs) {
    ok = c < P.n_contigs;
    if (ok) {
      o = __ldg(P.off + c);
      l = __ldg(P.len + c);
    }
  }
  const uint64_t eh = (uint64_t)e + P.closed;
  ok = ok && s <= e && eh <= l && o + eh <= kU32Max;
  bad += ok ? 0u : 1u;
  return ok ? make_uint2((uint32_t)(o + s), (uint32_t)(o + eh)) : make_uint2(kU32Max, 0u);
}

template <bool kVec>
__global__ void __launch_bounds__(kProjBlock) k_project(ProjArgs P) {
  uint32_t bad = 0;
  const uint64_t stride = (uint64_t)gridDim.x * kProjBlock;
  const uint64_t t0 = (uint64_t)blockIdx.x * kProjBlock + threadIdx.x;
  uint64_t tail_begin = 0;
  if (kVec) {
    const uint64_t n4 = P.n / 4;
    const uint4* S = reinterpret_cast<const uint4*>(P.start);
    const uint4* E = reinterpret_cast<const uint4*>(P.end);
    const uint4* Cc = reinterpret_cast<const uint4*>(P.chrom);
    uint4* O = reinterpret_cast<uint4*>(P.out);
    for (uint64_t q = t0; q < n4; q += stride) {
      const uint4 s = __ldcs(S + q), e = __ldcs(E + q);
      const uint4 c = P.n_contigs ? __ldcs(Cc + q) : make_uint4(0u, 0u, 0u, 0u);
      const uint2 r0 = project_one(P, c.x, s.x, e.x, bad);
      const uint2 r1 = project_one(P, c.y, s.y, e.y, bad);
      const uint2 r2 = project_one(P, c.z, s.z, e.z, bad);
      const uint2 r3 = project_one(P, c.w, s.w, e.w, bad);
      __stcs(O + 2 * q, make_uint4(r0.x, r0.y, r1.x, r1.y));
      __stcs(O + 2 * q + 1, make_uint4(r2.x, r2.y, r3.x, r3.y));
    }
    tail_begin = n4 * 4;
  }
  for (uint64_t i = tail_begin + t0; i < P.n; i += stride) {
    const uint32_t c = P.n_contigs ? P.chrom[i] : 0u;
    P.out[i] = project_one(P, c, P.start[i], P.end[i], bad);
  }
  if (P.n_rejected) {
    const uint32_t w = __reduce_add_sync(0xFFFFFFFFu, bad);
    if (lane_id() == 0 && w) atomicAdd(P.n_rejected, (unsigned long long)w);
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

bits_status launch_project(const uint32_t* d_chrom, const uint32_t* d_start, const uint32_t* d_end,
                           uint64_t n, const uint32_t* d_off, const uint32_t* d_len,
                           uint32_t n_contigs, bool closed, uint32_t* d_out,
                           uint64_t* d_n_rejected, cudaStream_t st) {
  if (d_n_rejected)
    BITS_CUDA_TRY(cudaMemsetAsync(d_n_rejected, 0, sizeof(uint64_t), st));
  if (n == 0) return BITS_OK;
  ProjArgs P{d_chrom, d_start, d_end, n, d_off, d_len, n_contigs, closed ? 1u : 0u,
             reinterpret_cast<uint2*>(d_out),
             reinterpret_cast<unsigned long long*>(d_n_rejected)};
  const bool vec = aligned16(d_start) && aligned16(d_end) && aligned16(d_out) &&
                   (n_contigs == 0 || aligned16(d_chrom));
  const uint64_t per_thread = vec ? 4 : 1;
  const uint64_t want = (n + per_thread * kProjBlock - 1) / (per_thread * kProjBlock);
  const uint32_t cap = (uint32_t)sm_count() * (2048 / kProjBlock);
  const uint32_t grid = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(want, 1), cap);
  if (vec)
    k_project<true><<<grid, kProjBlock, 0, st>>>(P);
  else
    k_project<false><<<grid, kProjBlock, 0, st>>>(P);
  BITS_LAUNCH_CHECK("k_project");
  return BITS_OK;
}

}  // namespace bits
