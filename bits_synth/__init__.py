"""Seeded synthetic genome-interval workloads.

This module only draws coordinates.  It holds none of the interval
intersection arithmetic (no counting, no searching of a database, no
shuffling): both the CUDA library's callers and the CPU oracle's callers feed
it the same seeds and get the same arrays, and each side then computes on its
own.

Every interval set is returned as an ``(n, 2)`` ``numpy.uint32`` array in
array-of-structures order ``[[start, end], ...]`` with half-open ``[start,
end)`` semantics, already projected onto one genome-wide coordinate line by
adding each contig's offset (the projection paragraph of the paper's Sec.
"BITS Algorithm", "The BITS solution to the counting problem").

Workload shapes (the paper's datasets are not available, so these stand in):

* ``config1``    one 1 Mbp contig, 10k queries x 10k database intervals.
* ``config2``    exome-vs-reads shape: 24 contigs, 200k queries, 20M reads
                 drawn 70 % from 200k Gaussian hotspots.
* ``config3``    Monte-Carlo significance shape (Table 1's 1e5/1e6 corner).
* ``config4``    learned-index scale: 100M x 100M on a 3.0 Gbp line.
* ``config5``    all-pairs screen shape (Sec. "Novel genomic
                 relationships"): 64 query sets x 32 database sets of
                 log-uniform size.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

U32_MAX = 2**32 - 1


@dataclass(frozen=True)
class Genome:
    """Contig table of a synthetic genome (offsets are cumulative lengths)."""

    offsets: np.ndarray  # uint32 [n_contigs], offset of each contig on the line
    lengths: np.ndarray  # uint32 [n_contigs]
    size: int            # sum of lengths (< 2**32)

    @property
    def n_contigs(self) -> int:
        return int(self.lengths.shape[0])


def make_genome(n_contigs: int = 24, lo: int = 50_000_000, hi: int = 250_000_000,
                seed: int = 3) -> Genome:
    """Contig lengths uniform integer in [lo, hi]; fails loudly past 2**32."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(lo, hi + 1, size=n_contigs, dtype=np.int64)
    size = int(lens.sum())
    if size > U32_MAX:
        raise OverflowError(f"genome of {size} bp does not fit uint32 coordinates "
                            f"(seed {seed}); choose another seed")
    offs = np.zeros(n_contigs, dtype=np.int64)
    offs[1:] = np.cumsum(lens)[:-1]
    return Genome(offs.astype(np.uint32), lens.astype(np.uint32), size)


def single_contig(length: int) -> Genome:
    return Genome(np.zeros(1, np.uint32), np.array([length], np.uint32), int(length))


def _pack(starts: np.ndarray, lens: np.ndarray) -> np.ndarray:
    starts = starts.astype(np.int64)
    ends = starts + lens.astype(np.int64)
    if starts.size and (starts.min() < 0 or ends.max() > U32_MAX):
        raise OverflowError("interval outside uint32 coordinate range")
    out = np.empty((starts.shape[0], 2), dtype=np.uint32)
    out[:, 0] = starts
    out[:, 1] = ends
    return out


def _contig_of(genome: Genome, g: np.ndarray) -> np.ndarray:
    """Contig index of genome-wide positions (generator bookkeeping only)."""
    return np.searchsorted(genome.offsets.astype(np.int64), g, side="right") - 1


def place_uniform(rng: np.random.Generator, genome: Genome, lens: np.ndarray) -> np.ndarray:
    """Genome-wide starts, contig chosen by length, position uniform inside it.

    The interval never crosses its contig's end: local start is uniform
    integer in [0, contig_len - len].
    """
    n = lens.shape[0]
    clen = genome.lengths.astype(np.int64)
    contig = rng.choice(genome.n_contigs, size=n, p=clen / clen.sum())
    hi = clen[contig] - lens.astype(np.int64)  # inclusive upper bound, >= 0
    if n and hi.min() < 0:
        raise ValueError("interval longer than its contig")
    local = rng.integers(0, hi + 1)
    return genome.offsets.astype(np.int64)[contig] + local


def make_hotspots(rng: np.random.Generator, genome: Genome, n_hot: int):
    """Hotspot centres uniform genome-wide, returned as (contig, local pos)."""
    g = rng.integers(0, genome.size, size=n_hot, dtype=np.int64)
    contig = _contig_of(genome, g)
    return contig, g - genome.offsets.astype(np.int64)[contig]


def place_hotspot(rng: np.random.Generator, genome: Genome, lens: np.ndarray,
                  hot_contig: np.ndarray, hot_pos: np.ndarray, sigma: float) -> np.ndarray:
    """Starts drawn N(centre, sigma) around a uniformly chosen hotspot.

    Rounded to nearest, then clamped so the interval stays inside the
    hotspot's contig.
    """
    n = lens.shape[0]
    h = rng.integers(0, hot_contig.shape[0], size=n)
    c = hot_contig[h]
    local = np.rint(rng.normal(hot_pos[h].astype(np.float64), sigma)).astype(np.int64)
    hi = genome.lengths.astype(np.int64)[c] - lens.astype(np.int64)
    local = np.clip(local, 0, hi)
    return genome.offsets.astype(np.int64)[c] + local


def clustered(rng: np.random.Generator, genome: Genome, lens: np.ndarray, n_hot: int,
              sigma: float = 200.0, frac_hot: float = 0.7) -> np.ndarray:
    """frac_hot of the intervals around n_hot hotspots, the rest uniform."""
    n = lens.shape[0]
    hot_contig, hot_pos = make_hotspots(rng, genome, n_hot)
    is_hot = rng.random(n) < frac_hot
    starts = np.empty(n, dtype=np.int64)
    starts[is_hot] = place_hotspot(rng, genome, lens[is_hot], hot_contig, hot_pos, sigma)
    starts[~is_hot] = place_uniform(rng, genome, lens[~is_hot])
    return _pack(starts, lens)


def log_uniform_int(rng: np.random.Generator, lo: float, hi: float, n: int) -> np.ndarray:
    """round(exp(U(ln lo, ln hi)))."""
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))).astype(np.int64)


# --------------------------------------------------------------------------- configs

def config1(n_a: int = 10_000, n_b: int = 10_000, contig_len: int = 1_000_000,
            seed_a: int = 1, seed_b: int = 2):
    """One contig; lengths U[50,500]; starts uniform on [0, contig_len - len)."""
    def draw(seed, n):
        rng = np.random.default_rng(seed)
        lens = rng.integers(50, 501, size=n, dtype=np.int64)
        starts = rng.integers(0, contig_len - lens)  # exclusive high
        return _pack(starts, lens)
    return draw(seed_a, n_a), draw(seed_b, n_b)


def config2(n_a: int = 200_000, n_b: int = 20_000_000, n_hot: int = 200_000,
            genome: Genome | None = None, seed_a: int = 4, seed_b: int = 5):
    """Exome-vs-reads shape on the 24-contig genome.

    A: lengths round(N(150, 30)) clipped to [50, 400], placed uniformly.
    B: reads of length 100, 70 % from n_hot Gaussian hotspots (sigma 200 bp).
    """
    genome = genome or make_genome()
    rng = np.random.default_rng(seed_a)
    la = np.clip(np.rint(rng.normal(150.0, 30.0, size=n_a)), 50, 400).astype(np.int64)
    a = _pack(place_uniform(rng, genome, la), la)
    rng = np.random.default_rng(seed_b)
    lb = np.full(n_b, 100, dtype=np.int64)
    b = clustered(rng, genome, lb, n_hot)
    return genome, a, b


def config3(n_a: int = 100_000, n_b: int = 1_000_000, n_hot: int = 200_000,
            genome: Genome | None = None, seed_a: int = 8, seed_b: int = 9):
    """Monte-Carlo shape: A uniform, B clustered; lengths U[100, 2000]."""
    genome = genome or make_genome()
    rng = np.random.default_rng(seed_a)
    la = rng.integers(100, 2001, size=n_a, dtype=np.int64)
    a = _pack(place_uniform(rng, genome, la), la)
    rng = np.random.default_rng(seed_b)
    lb = rng.integers(100, 2001, size=n_b, dtype=np.int64)
    b = clustered(rng, genome, lb, n_hot)
    return genome, a, b


def config4(n_a: int = 100_000_000, n_b: int = 100_000_000, space: int = 3_000_000_000,
            n_mix: int = 1000, seed_a: int = 12, seed_b: int = 13, seed_mix: int = 14):
    """Learned-index scale on one 3.0 Gbp line.

    B: 80 % from an equal-weight mixture of n_mix Gaussians (centres U[0,
    space), sigma U[1e3, 1e6]), 20 % uniform; lengths log-uniform [50, 1e4].
    A: lengths log-uniform [50, 1e4], placed uniformly.
    """
    rng = np.random.default_rng(seed_mix)
    centres = rng.uniform(0.0, float(space), size=n_mix)
    sigmas = rng.uniform(1e3, 1e6, size=n_mix)

    rng = np.random.default_rng(seed_b)
    lb = log_uniform_int(rng, 50, 10_000, n_b)
    hi_b = space - lb
    mix = rng.random(n_b) < 0.8
    sb = np.empty(n_b, dtype=np.int64)
    k = int(mix.sum())
    comp = rng.integers(0, n_mix, size=k)
    sb[mix] = np.rint(rng.normal(centres[comp], sigmas[comp])).astype(np.int64)
    sb[~mix] = rng.integers(0, hi_b[~mix] + 1)
    sb = np.clip(sb, 0, hi_b)
    b = _pack(sb, lb)
    del sb, mix, comp

    rng = np.random.default_rng(seed_a)
    la = log_uniform_int(rng, 50, 10_000, n_a)
    sa = rng.integers(0, space - la + 1)
    a = _pack(sa, la)
    return a, b


def config5_sizes(n_sets_a: int = 64, n_sets_b: int = 32, lo: float = 1_000,
                  hi: float = 20_000_000, seed: int = 11):
    rng = np.random.default_rng(seed)
    sizes = log_uniform_int(rng, lo, hi, n_sets_a + n_sets_b)
    return sizes[:n_sets_a], sizes[n_sets_a:]


def config5_set(index: int, size: int, genome: Genome, seed: int = 11) -> np.ndarray:
    """One set of the all-pairs screen (index < n_sets_a: query set).

    Lengths U[50, 5000]; even-indexed sets clustered around max(1, n/100)
    hotspots (sigma 200 bp, 70 %), odd-indexed sets uniform.
    """
    ss = np.random.SeedSequence([seed, index])
    rng = np.random.default_rng(ss)
    lens = rng.integers(50, 5001, size=int(size), dtype=np.int64)
    if index % 2 == 0:
        return clustered(rng, genome, lens, max(1, int(size) // 100))
    return _pack(place_uniform(rng, genome, lens), lens)


def config5(n_sets_a: int = 64, n_sets_b: int = 32, lo: float = 1_000, hi: float = 20_000_000,
            seed: int = 11, genome: Genome | None = None):
    """All-pairs screen shape: lists of query sets and database sets."""
    genome = genome or make_genome()
    sa, sb = config5_sizes(n_sets_a, n_sets_b, lo, hi, seed)
    a_sets = [config5_set(i, int(s), genome, seed) for i, s in enumerate(sa)]
    b_sets = [config5_set(n_sets_a + j, int(s), genome, seed) for j, s in enumerate(sb)]
    return genome, a_sets, b_sets


# ----------------------------------------------------------------- edge-case inputs

def tiny_random(seed: int, n_a: int, n_b: int, coord_max: int = 64, max_len: int = 8,
                allow_empty_queries: bool = True):
    """Small dense sets with many ties, duplicates and touching endpoints."""
    rng = np.random.default_rng(seed)
    def draw(n, min_len):
        lens = rng.integers(min_len, max(min_len, min(max_len, coord_max)) + 1, size=n,
                            dtype=np.int64)
        starts = rng.integers(0, coord_max - lens + 1)
        return _pack(starts, lens)
    return draw(n_a, 0 if allow_empty_queries else 1), draw(n_b, 1)


def nested(m: int, base: int = 0) -> np.ndarray:
    """m intervals each containing the next: [base+i, base+2m-i), i = 0..m-1."""
    i = np.arange(m, dtype=np.int64)
    return _pack(base + i, 2 * m - 2 * i)


def unit_tiles(m: int, base: int = 0) -> np.ndarray:
    """m unit intervals [base+i, base+i+1)."""
    return _pack(base + np.arange(m, dtype=np.int64), np.ones(m, dtype=np.int64))


def mc_contig_table(genome: Genome):
    """(offsets, lengths) as uint32 arrays, the form the MC calls take."""
    return genome.offsets.copy(), genome.lengths.copy()


def local_intervals(genome: Genome, n: int, seed: int, lo: int = 50, hi: int = 400,
                    closed: bool = False, bad_frac: float = 0.0):
    """Chromosome-local intervals in the form a BED file holds them.

    Returns uint32 arrays (contig id, start, end).  The chromosome is chosen
    with probability proportional to its length and the start is uniform
    over the positions where an interval of length U[lo, hi] fits; for
    closed output the end is start + length - 1.  A fraction ``bad_frac`` of
    rows is then spoiled in one of three ways picked at random: a contig id
    past the table, a start after the end, or an end past the contig.
    """
    rng = np.random.default_rng(seed)
    lens = rng.integers(lo, hi + 1, size=n, dtype=np.int64)
    clen = genome.lengths.astype(np.int64)
    contig = rng.choice(genome.n_contigs, size=n, p=clen / clen.sum())
    start = rng.integers(0, clen[contig] - lens + 1)
    end = start + lens - (1 if closed else 0)
    if bad_frac > 0 and n:
        bad = np.flatnonzero(rng.random(n) < bad_frac)
        kind = rng.integers(0, 3, size=bad.shape[0])
        k0, k1, k2 = bad[kind == 0], bad[kind == 1], bad[kind == 2]
        contig[k0] = genome.n_contigs + rng.integers(0, 1000, size=k0.shape[0])
        start[k1] = end[k1] + rng.integers(1, 50, size=k1.shape[0])
        end[k2] = clen[contig[k2]] + rng.integers(0, 50, size=k2.shape[0])
    return contig.astype(np.uint32), start.astype(np.uint32), end.astype(np.uint32)
