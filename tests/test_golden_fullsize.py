"""The full-size expected values under tests/golden/ are the oracle's.

make_fullsize.py writes the 10,000 Monte-Carlo totals and the 64 x 32
all-pairs matrix from the oracle alone; the GPU tests compare the library
with them entry by entry.  Here (CPU only, a few seconds) the stored values
are tied back to the oracle and to what the definitions fix: the tally and
p-value follow from the stored totals, the observed total and a sample of
shuffles and matrix entries are recomputed by the oracle, and every total
respects 0 <= T <= |A| |B|.
"""
import numpy as np
import pytest

import bits_synth as synth
import goldens
import oracle

O = oracle.get()


def test_mc_golden_is_consistent_and_matches_oracle_sample():
    obs, k, (pnum, pden), totals = goldens.read_mc_fullsize()
    assert totals.shape == (10_000,)
    assert k == int((totals >= np.uint64(obs)).sum())          # Sec. "Monte Carlo Simulations" tally
    assert (pnum, pden) == (k + 1, 10_001)
    genome, a, b = synth.config3()
    assert int(totals.max()) <= a.shape[0] * b.shape[0]
    co, cl = synth.mc_contig_table(genome)
    bs, be = O.build(b)
    assert O.count_sorted(a, bs, be, threads=8, want_counts=False)[1] == obs
    for s in (0, 1, 255, 256, 4321, 9983, 9984, 9999):
        t, *_ = O.mc(a, co, cl, bs, be, seed=7, s_begin=s, s_end=s + 1, threads=8)
        assert int(t[0]) == int(totals[s]), s


def test_allpairs_golden_matches_oracle_sample():
    m = goldens.read_allpairs_fullsize()
    assert m.shape == (64, 32)
    sizes_a, sizes_b = synth.config5_sizes()
    assert (m <= np.outer(sizes_a, sizes_b).astype(np.uint64)).all()
    genome = synth.make_genome()
    small_a = [int(i) for i in np.argsort(sizes_a)[:3]]
    a_sets = {i: synth.config5_set(i, int(sizes_a[i]), genome) for i in small_a}
    for j in [int(x) for x in np.argsort(sizes_b)[:3]] + [int(np.argmax(sizes_b))]:
        bs, be = O.build(synth.config5_set(len(sizes_a) + j, int(sizes_b[j]), genome))
        for i in small_a:
            assert O.count_sorted(a_sets[i], bs, be, want_counts=False)[1] == int(m[i, j]), (i, j)
