"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Every oracle function is checked here against at least one of: a hand-worked
fixture (tests/golden), a closed form, an invariant of the definition, a
published known-answer vector, exact big-integer arithmetic, or brute force
over all pairs.  test_mutants_fail_pins recompiles the oracle with planted
mistakes and checks that these pins catch each one.
"""
import os
import tempfile

import numpy as np
import pytest

import bits_synth as synth
import oracle
from goldens import (read_count_fixture, read_enumerate_fixture, read_mc_summary_fixture,
                     read_philox_kat, read_projection_fixture)

O = oracle.get()


# ---------------------------- counting (Sec. "Interval Set Intersection problem", Alg. 1, 2)

@pytest.mark.parametrize("name", ["containment.txt", "duplicates.txt"])
def test_golden_fixture(name):
    a, b, exp, total = read_count_fixture(name)
    c, t = O.count_brute(a, b)
    np.testing.assert_array_equal(c, exp)
    assert t == total
    c2, t2 = O.count(a, b)
    np.testing.assert_array_equal(c2, exp)
    assert t2 == total


def test_closed_form_unit_tiles():
    m = 50
    b = synth.unit_tiles(m)
    rng = np.random.default_rng(0)
    s = rng.integers(0, 70, size=400)
    e = s + rng.integers(0, 20, size=400)
    a = np.stack([s, e], 1).astype(np.uint32)
    expect = np.maximum(0, np.minimum(e, m) - np.maximum(s, 0))
    expect[s == e] = 0
    for fn in (O.count_brute, O.count):
        c, t = fn(a, b)
        np.testing.assert_array_equal(c, expect)
        assert t == int(expect.sum())


def test_closed_form_nested():
    # [i, 2m-i) for i < m; the point query [x, x+1) meets min(x+1, 2m-x) of them.
    m = 40
    b = synth.nested(m)
    x = np.arange(0, 2 * m + 5)
    a = np.stack([x, x + 1], 1).astype(np.uint32)
    expect = np.clip(np.minimum(x + 1, 2 * m - x), 0, m)
    for fn in (O.count_brute, O.count):
        c, _ = fn(a, b)
        np.testing.assert_array_equal(c, expect)


def test_all_of_b_in_one_interval():
    b = np.array([[0, 1000]] * 7 + [[10, 20]], np.uint32)
    a = np.array([[500, 501], [15, 15], [0, 0], [1000, 1001], [999, 1000]], np.uint32)
    c, _ = O.count(a, b)
    np.testing.assert_array_equal(c, [7, 8, 0, 0, 7])


def test_sorted_matches_brute_tiny_random():
    for seed in range(400):
        rng = np.random.default_rng(seed)
        na, nb = int(rng.integers(0, 30)), int(rng.integers(0, 30))
        a, b = synth.tiny_random(seed, na, nb, coord_max=int(rng.integers(2, 80)),
                                 max_len=int(rng.integers(1, 12)))
        c1, t1 = O.count_brute(a, b)
        c2, t2 = O.count(a, b)
        np.testing.assert_array_equal(c1, c2)
        assert t1 == t2 == int(c1.sum())
        assert (c1 <= nb).all()


def test_invariants():
    rng = np.random.default_rng(7)
    for seed in range(60):
        a, b = synth.tiny_random(1000 + seed, 25, 30, coord_max=200, max_len=30,
                                 allow_empty_queries=False)
        _, t_ab = O.count(a, b)
        _, t_ba = O.count(b, a)
        assert t_ab == t_ba                                   # symmetric predicate
        shift = int(rng.integers(1, 1 << 30))
        _, t_sh = O.count(a + np.uint32(shift), b + np.uint32(shift))
        assert t_sh == t_ab                                   # translation invariance
        far = b + np.uint32(10_000)
        _, t_far = O.count(a, far)
        assert t_far == 0                                     # disjoint contigs
        k = int(rng.integers(1, b.shape[0]))
        _, t1 = O.count(a, b[:k])
        _, t2 = O.count(a, b[k:])
        assert t1 + t2 == t_ab                                # additive over splits of B
        k = int(rng.integers(1, a.shape[0]))
        _, t3 = O.count(a[:k], b)
        _, t4 = O.count(a[k:], b)
        assert t3 + t4 == t_ab                                # additive over splits of A
        c, _ = O.count(a, b)
        assert ((c > 0).any()) == (t_ab > 0)                  # decision problem


def test_total_from_each_side_sorted_keys():
    """The rank-sum identity the all-pairs count from databases relies on:
    summed over A, Algorithm 2's ICount needs each sorted array only on its
    own, total(A, B) = sum_{x in A_E} #(B_S < x) - sum_{x in A_S} #(B_E <= x),
    and the same pairs counted from B's side give the mirror image.  Checked
    against the oracle's brute force (numpy's searchsorted gives the ranks)."""
    for seed in range(40):
        a, b = synth.tiny_random(2000 + seed, 37, 23, coord_max=300, max_len=40,
                                 allow_empty_queries=False)
        _, brute = O.count_brute(a, b)
        a_s, a_e = np.sort(a[:, 0]), np.sort(a[:, 1])
        b_s, b_e = np.sort(b[:, 0]), np.sort(b[:, 1])
        from_a = int(np.searchsorted(b_s, a_e, side="left").sum()) - \
            int(np.searchsorted(b_e, a_s, side="right").sum())
        from_b = int(np.searchsorted(a_s, b_e, side="left").sum()) - \
            int(np.searchsorted(a_e, b_s, side="right").sum())
        assert from_a == brute and from_b == brute
        # the k-th sorted start and end of one side form a valid search pair
        assert (a_s < a_e).all() and (b_s < b_e).all()


def test_config1_full_brute_force():
    a, b = synth.config1()
    c1, t1 = O.count_brute(a, b)
    c2, t2 = O.count(a, b)
    np.testing.assert_array_equal(c1, c2)
    assert t1 == t2


def test_threads_do_not_change_result():
    _, a, b = synth.config2(n_a=20_000, n_b=200_000, n_hot=2000)
    bs, be = O.build(b)
    c1, t1 = O.count_sorted(a, bs, be, threads=1)
    c4, t4 = O.count_sorted(a, bs, be, threads=4)
    np.testing.assert_array_equal(c1, c4)
    assert t1 == t4


def test_build_is_sorted_permutation():
    b = synth.config1()[1]
    bs, be = O.build(b)
    assert (np.diff(bs.astype(np.int64)) >= 0).all() and (np.diff(be.astype(np.int64)) >= 0).all()
    np.testing.assert_array_equal(np.sort(b[:, 0]), bs)
    np.testing.assert_array_equal(np.sort(b[:, 1]), be)


def test_rejects_bad_input():
    good = np.array([[1, 5]], np.uint32)
    with pytest.raises(ValueError):
        O.count(np.array([[5, 4]], np.uint32), good)        # inverted query
    with pytest.raises(ValueError):
        O.count(good, np.array([[3, 3]], np.uint32))        # empty database interval
    with pytest.raises(ValueError):
        O.mc_place(np.array([[95, 105]], np.uint32), [0, 100], [100, 100], 1, 0)  # crosses contig


def test_extreme_coordinates():
    top = 2**32 - 1
    b = np.array([[top - 5, top], [0, 1], [top - 1, top]], np.uint32)
    a = np.array([[top - 1, top - 1], [top - 2, top], [top, top], [0, 0], [0, top]], np.uint32)
    c1, _ = O.count_brute(a, b)
    c2, _ = O.count(a, b)
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(c1, [1, 2, 0, 0, 3])


# ------------------------------------------------------------------ Philox and the position map

def test_philox_known_answers():
    for ctr, key, expect in read_philox_kat():
        np.testing.assert_array_equal(O.philox(ctr, key), np.array(expect, np.uint32))


def test_scale_matches_exact_integer_arithmetic():
    rng = np.random.default_rng(3)
    cases = [(0, 1), (2**64 - 1, 1), (2**64 - 1, 2**32), (2**63, 3), (1, 2**33)]
    for _ in range(2000):
        cases.append((int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2)),
                      int(rng.integers(1, 2**32 + 1))))
    for u, n in cases:
        assert O.scale_u64(u, n) == (u * n) >> 64


def test_mc_place_pinned_by_known_answer():
    # Interval 0 of shuffle 0 with seed 0 draws Philox(ctr 0, key 0), the first
    # known-answer vector: x0 = 6627e8d5, x1 = e169c58d.
    u = (0xE169C58D << 32) | 0x6627E8D5
    off, ln = [0, 1000], [1000, 5000]
    for length, contig in ((10, 0), (123, 1), (1000, 0)):
        start = off[contig] + 7 if length < 1000 else off[contig]
        a = np.array([[start, start + length]], np.uint32)
        out = O.mc_place(a, off, ln, seed=0, s=0)
        expect = off[contig] + ((u * (ln[contig] - length + 1)) >> 64)
        assert int(out[0, 0]) == expect and int(out[0, 1]) == expect + length


def test_mc_place_invariants():
    genome, a, _ = synth.config3(n_a=5000, n_b=10)
    co, cl = synth.mc_contig_table(genome)
    contig_before = np.searchsorted(co, a[:, 0], side="right") - 1
    for s in (0, 1, 77, 9999):
        p = O.mc_place(a, co, cl, seed=7, s=s)
        np.testing.assert_array_equal(p[:, 1] - p[:, 0], a[:, 1] - a[:, 0])   # length kept
        c = np.searchsorted(co, p[:, 0], side="right") - 1
        np.testing.assert_array_equal(c, contig_before)                       # contig kept
        assert (p[:, 1].astype(np.int64) <= co[c].astype(np.int64) + cl[c]).all()  # inside it
    assert not np.array_equal(O.mc_place(a, co, cl, 7, 0), O.mc_place(a, co, cl, 7, 1))


def test_mc_place_uniform_chi_square():
    # One interval, 20000 shuffles, range 1000: 10 equal bins of offsets.
    a = np.array([[100, 101]], np.uint32)
    co, cl = np.array([0], np.uint32), np.array([1000], np.uint32)
    offs = np.array([int(O.mc_place(a, co, cl, seed=12345, s=s)[0, 0]) for s in range(20000)])
    hist = np.bincount(offs // 100, minlength=10)
    chi2 = float((((hist - 2000.0) ** 2) / 2000.0).sum())
    assert chi2 < 37.0   # chi-square with 9 dof, p about 4e-5


def test_mc_fixed_placement_closed_form():
    # Contigs exactly as long as their interval: every shuffle puts it at the
    # contig start, so every total equals the count of A moved to contig starts.
    co = np.array([0, 100, 300], np.uint32)
    cl = np.array([100, 200, 50], np.uint32)
    a = np.array([[10, 110 - 10], [150, 350], [320, 330]], np.uint32)
    a[0] = [0, 100]
    a[1] = [100, 300]
    a[2] = [300, 350]
    b = np.array([[50, 60], [99, 101], [299, 301], [340, 345], [0, 400]], np.uint32)
    bs, be = O.build(b)
    totals, obs, k, p = O.mc(a, co, cl, bs, be, seed=5, s_begin=0, s_end=16)
    _, expect = O.count_brute(a, b)
    assert (totals == expect).all() and obs == expect
    assert k == 16 and p == 1.0


def test_mc_tally_and_pvalue():
    genome, a, b = synth.config3(n_a=300, n_b=3000, n_hot=50)
    co, cl = synth.mc_contig_table(genome)
    bs, be = O.build(b)
    totals, obs, k, p = O.mc(a, co, cl, bs, be, seed=7, s_begin=0, s_end=64)
    _, obs_brute = O.count_brute(a, b)
    assert obs == obs_brute
    assert k == int((totals >= obs).sum())
    assert p == (k + 1) / 65.0 and 1 / 65.0 <= p <= 1.0
    for s in (0, 13, 63):                                   # each total is a recount
        _, t = O.count_brute(O.mc_place(a, co, cl, 7, s), b)
        assert totals[s] == t
    t_lo, *_ = O.mc(a, co, cl, bs, be, seed=7, s_begin=0, s_end=20)   # resumable by range
    t_hi, *_ = O.mc(a, co, cl, bs, be, seed=7, s_begin=20, s_end=64)
    np.testing.assert_array_equal(np.concatenate([t_lo, t_hi]), totals)
    t_mt, *_ = O.mc(a, co, cl, bs, be, seed=7, s_begin=0, s_end=64, threads=4)
    np.testing.assert_array_equal(t_mt, totals)
    # Observed beyond every shuffle: p is the smallest possible value.
    empty = np.zeros(0, np.uint32)
    tz, oz, kz, pz = O.mc(a, co, cl, empty, empty, seed=7, s_begin=0, s_end=9)
    assert (tz == 0).all() and oz == 0 and kz == 9 and pz == 1.0


# ------------------- enumeration (Sec. "Interval Set Intersection problem", "BITS Algorithm")

def _partners(off, pairs, i):
    return [int(x) for x in pairs[int(off[i]):int(off[i + 1]), 1]]


def test_enumerate_golden():
    a, b, exp, total, scan_lists = read_enumerate_fixture()
    for fn, ordered in ((O.enumerate_scan, True), (O.enumerate_brute, False)):
        off, pairs = fn(a, b)
        assert int(off[-1]) == total == pairs.shape[0]
        np.testing.assert_array_equal(np.diff(off.astype(np.int64)), exp)
        for i, want in enumerate(scan_lists):
            got = _partners(off, pairs, i)
            assert got == (want if ordered else sorted(want)), (fn.__name__, i)
            assert (pairs[int(off[i]):int(off[i + 1]), 0] == i).all()


@pytest.mark.parametrize("seed", range(40))
def test_enumerate_scan_matches_definition(seed):
    a, b = synth.tiny_random(seed, n_a=60, n_b=80, coord_max=200, max_len=40)
    ob, pb = O.enumerate_brute(a, b)
    os_, ps = O.enumerate_scan(a, b)
    np.testing.assert_array_equal(ob, os_)
    counts, _ = O.count_brute(a, b)
    np.testing.assert_array_equal(np.diff(ob.astype(np.int64)), counts)
    bstart = b[:, 0].astype(np.int64)
    for i in range(a.shape[0]):
        got = _partners(os_, ps, i)
        assert sorted(got) == _partners(ob, pb, i)
        # scan order: descending start, equal starts in descending index
        keys = [(-bstart[j], -j) for j in got]
        assert keys == sorted(keys)


def test_enumerate_nested_closed_form():
    # [i, 2m-i) for i < m: the point query [x, x+1) meets min(x+1, 2m-x) of
    # them, the innermost ones; the scan walks past none of the others.
    m = 30
    b = synth.nested(m)
    x = np.arange(0, 2 * m + 3)
    a = np.stack([x, x + 1], 1).astype(np.uint32)
    off, pairs = O.enumerate_scan(a, b)
    for i, xi in enumerate(x):
        want = set(range(0, min(xi + 1, 2 * m - xi))) if xi < 2 * m else set()
        assert set(_partners(off, pairs, i)) == want


# -- MC summary, per-set streams (Sec. "Monte Carlo Simulations", "Novel genomic relationships")

def _score_ok(got: float, spec: str) -> bool:
    import math
    from fractions import Fraction
    if spec == "nan":
        return math.isnan(got)
    if spec in ("inf", "-inf"):
        return got == float(spec)
    r = Fraction(spec)
    return got == math.log2(r.numerator / r.denominator)


def test_mc_summary_golden():
    for obs, totals, exp in read_mc_summary_fixture():
        got = O.mc_summary(totals, obs)
        for k in ("k_ge", "k_le", "median_lo", "median_hi"):
            assert got[k] == exp[k], (obs, list(totals), k)
        assert got["p_enrich"] == exp["p_enrich"].numerator / exp["p_enrich"].denominator
        assert got["p_deplete"] == exp["p_deplete"].numerator / exp["p_deplete"].denominator
        assert _score_ok(got["log2_enrichment"], exp["score"]), (obs, list(totals))


@pytest.mark.parametrize("n", [1, 2, 7, 100, 10_000, 10_001])
def test_mc_summary_properties(n):
    rng = np.random.default_rng(n)
    t = rng.integers(1000, 1100, size=n).astype(np.uint64)
    obs = int(rng.integers(990, 1110))
    got = O.mc_summary(t, obs)
    # Library median (mean of the two middles for even n) and counting identities.
    assert (got["median_lo"] + got["median_hi"]) / 2 == np.median(t.astype(np.float64))
    assert got["median_lo"] <= got["median_hi"]
    assert got["k_ge"] + got["k_le"] == n + int((t == obs).sum())
    assert got["k_ge"] == int((t >= obs).sum())
    # Shuffle order does not matter.
    got2 = O.mc_summary(rng.permutation(t), obs)
    assert got2 == got or (np.isnan(got["log2_enrichment"]) and np.isnan(got2["log2_enrichment"]))
    # The score doubles the ratio when observed doubles: log2 grows by exactly 1
    # whenever the ratio stays in the normal double range.
    g4 = O.mc_summary(t, 2 * obs)
    assert g4["log2_enrichment"] == pytest.approx(got["log2_enrichment"] + 1.0, abs=1e-12)


def test_mc_summary_empty_and_overflow():
    got = O.mc_summary(np.zeros(0, np.uint64), 7)
    assert got["k_ge"] == 0 and got["p_enrich"] == 1.0 and got["p_deplete"] == 1.0
    with pytest.raises(ValueError):
        O.mc_summary(np.array([2**63, 2**63], np.uint64), 1)


def test_mc_set_index_streams():
    # Set 0 is the single test's stream (pinned by the known-answer placement);
    # set i reads its Philox block at counter word 2 = i.
    genome = synth.single_contig(1000)
    co, cl = synth.mc_contig_table(genome)
    a = np.array([[7, 17], [100, 140], [0, 1000]], np.uint32)
    np.testing.assert_array_equal(O.mc_place(a, co, cl, 9, 4), O.mc_place(a, co, cl, 9, 4, 0))
    for set_index in (1, 5, 2**31 + 3):
        out = O.mc_place(a, co, cl, seed=9, s=4, set_index=set_index)
        for k in range(a.shape[0]):
            x = O.philox([k, 4, set_index, 0], [9, 0])
            u = (int(x[1]) << 32) | int(x[0])
            ln = int(a[k, 1] - a[k, 0])
            start = (u * (1000 - ln + 1)) >> 64
            assert (int(out[k, 0]), int(out[k, 1])) == (start, start + ln)
        assert not np.array_equal(out[:2], O.mc_place(a, co, cl, 9, 4)[:2])
    # Totals of set i are recounts of set i's placements.
    g3, a3, b3 = synth.config3(n_a=200, n_b=2000, n_hot=40)
    co3, cl3 = synth.mc_contig_table(g3)
    bs, be = O.build(b3)
    tot, obs, _, _ = O.mc(a3, co3, cl3, bs, be, seed=3, s_begin=2, s_end=6, set_index=7)
    for j, s_ in enumerate(range(2, 6)):
        _, t = O.count_brute(O.mc_place(a3, co3, cl3, 3, s_, 7), b3)
        assert tot[j] == t


# ------ projection, closed intervals (Sec. "Interval Set Intersection problem", "BITS Algorithm")

def _expected_rows(rows):
    return np.array([r if r is not None else (0xFFFFFFFF, 0) for r in rows], np.uint32), \
        sum(r is None for r in rows)


@pytest.mark.parametrize("closed", [False, True])
def test_projection_golden(closed):
    co, cl, chrom, s, e, ho, cc = read_projection_fixture()
    out, bad = O.project(chrom, s, e, co, cl, closed=closed)
    exp, nbad = _expected_rows(cc if closed else ho)
    np.testing.assert_array_equal(out, exp)
    assert bad == nbad


def test_closed_predicate_golden():
    # The printed predicate, brute force, against hand counts; then the same
    # sets mapped to half-open [s, e + 1) and counted by both half-open forms.
    a, b, exp, total = read_count_fixture("closed.txt")
    c, t = O.count_brute_closed(a, b)
    np.testing.assert_array_equal(c, exp)
    assert t == total
    pa, bad_a = O.project(None, a[:, 0], a[:, 1], closed=True)
    pb, bad_b = O.project(None, b[:, 0], b[:, 1], closed=True)
    assert bad_a == 0 and bad_b == 0
    for fn in (O.count_brute, O.count):
        c2, t2 = fn(pa, pb)
        np.testing.assert_array_equal(c2, exp)
        assert t2 == total


def _local_sets(rng, n, lens):
    chrom = rng.integers(0, len(lens), size=n)
    ln = 1 + (rng.random(n) * np.minimum(11, lens[chrom])).astype(np.int64)
    s = (rng.random(n) * (lens[chrom] - ln + 1)).astype(np.int64)
    return chrom, s, s + ln


@pytest.mark.parametrize("closed", [False, True])
def test_projection_matches_per_contig_brute_force(closed):
    # Intervals on different chromosomes never meet, and on the same one they
    # meet by the local predicate: counted here pair by pair on the local
    # coordinates, with no projection, and compared with counting the
    # projected sets on one line.
    rng = np.random.default_rng(5)
    lens = np.array([40, 7, 90, 25, 60], np.int64)
    off = np.concatenate([[0], np.cumsum(lens)[:-1]])
    ca, sa, ea = _local_sets(rng, 300, lens)
    cb, sb, eb = _local_sets(rng, 400, lens)
    if closed:                      # closed [s, e] with e = s + len - 1
        ea, eb = ea - 1, eb - 1
    same = ca[:, None] == cb[None, :]
    if closed:
        meet = (sa[:, None] <= eb[None, :]) & (ea[:, None] >= sb[None, :])
    else:
        meet = (sb[None, :] < ea[:, None]) & (eb[None, :] > sa[:, None])
    expect = (same & meet).sum(1)
    pa, bad_a = O.project(ca, sa, ea, off, lens, closed=closed)
    pb, bad_b = O.project(cb, sb, eb, off, lens, closed=closed)
    assert bad_a == 0 and bad_b == 0
    c, t = O.count(pa, pb)
    np.testing.assert_array_equal(c, expect)
    assert t == int(expect.sum())
    # Projected intervals stay inside their chromosome and keep their length.
    ln = (ea - sa) + (1 if closed else 0)
    assert (pa[:, 0] >= off[ca]).all() and (pa[:, 1] <= off[ca] + lens[ca]).all()
    np.testing.assert_array_equal(pa[:, 1].astype(np.int64) - pa[:, 0], ln)


def test_projection_rejects_and_edges():
    # No contig table: one line at offset 0 spanning 32 bits.
    top = 0xFFFFFFFF
    out, bad = O.project(None, [0, 0, 5, top], [top, top, 4, top], closed=False)
    np.testing.assert_array_equal(out, [[0, top], [0, top], [top, 0], [top, top]])
    assert bad == 1
    out, bad = O.project(None, [0, top - 1], [top, top - 1], closed=True)
    np.testing.assert_array_equal(out, [[top, 0], [top - 1, top]])
    assert bad == 1
    # A chromosome whose end reaches 2^32 - 1 exactly is usable; one past is not.
    out, bad = O.project([0, 0], [0, 0], [10, 11], [top - 10], [11], closed=False)
    np.testing.assert_array_equal(out, [[top - 10, top], [top, 0]])
    assert bad == 1
    out, bad = O.project([], [], [], [0], [5])
    assert out.shape == (0, 2) and bad == 0


# ------------------------------------------------------------------- planted mistakes

MUTANTS = ["ORACLE_MUTANT_CLOSED", "ORACLE_MUTANT_LAST_LOWER", "ORACLE_MUTANT_PHILOX",
           "ORACLE_MUTANT_SCALE", "ORACLE_MUTANT_WORD_ORDER", "ORACLE_MUTANT_TALLY",
           "ORACLE_MUTANT_PROJECT_OFFSET", "ORACLE_MUTANT_PROJECT_CLOSED",
           "ORACLE_MUTANT_BRUTE_CLOSED", "ORACLE_MUTANT_DEPLETE", "ORACLE_MUTANT_MEDIAN",
           "ORACLE_MUTANT_SET_WORD", "ORACLE_MUTANT_ENUM_END"]


def _pins_pass(o: oracle.Oracle) -> bool:
    try:
        for name in ("containment.txt", "duplicates.txt"):
            a, b, exp, total = read_count_fixture(name)
            c, t = o.count_brute(a, b)
            assert (c == exp).all() and t == total
            c, t = o.count(a, b)
            assert (c == exp).all() and t == total
        for ctr, key, expect in read_philox_kat():
            assert (o.philox(ctr, key) == np.array(expect, np.uint32)).all()
        u = (0xE169C58D << 32) | 0x6627E8D5
        out = o.mc_place(np.array([[7, 17]], np.uint32), [0], [1000], seed=0, s=0)
        assert int(out[0, 0]) == (u * 991) >> 64
        for uu, n in ((2**64 - 1, 2**32), (2**63, 3)):
            assert o.scale_u64(uu, n) == (uu * n) >> 64
        co = np.array([0], np.uint32)
        cl = np.array([10], np.uint32)
        aa = np.array([[0, 10]], np.uint32)
        bb = np.array([[2, 3]], np.uint32)
        bs, be = o.build(bb)
        tot, obs, k, p = o.mc(aa, co, cl, bs, be, seed=1, s_begin=0, s_end=4)
        assert k == 4 and p == 1.0
        co, cl, chrom, s, e, ho, cc = read_projection_fixture()
        for closed, rows in ((False, ho), (True, cc)):
            out, bad = o.project(chrom, s, e, co, cl, closed=closed)
            exp, nbad = _expected_rows(rows)
            assert (out == exp).all() and bad == nbad
        a, b, exp, total = read_count_fixture("closed.txt")
        c, t = o.count_brute_closed(a, b)
        assert (c == exp).all() and t == total
        for obs, totals, exp in read_mc_summary_fixture():
            got = o.mc_summary(totals, obs)
            assert all(got[k] == exp[k] for k in ("k_ge", "k_le", "median_lo", "median_hi"))
        x = o.philox([1, 4, 5, 0], [9, 0])
        u = (int(x[1]) << 32) | int(x[0])
        placed = o.mc_place(np.array([[3, 4], [0, 10]], np.uint32), [0], [1000], 9, 4, 5)
        assert int(placed[1, 0]) == (u * 991) >> 64
        a, b, exp, total, scan_lists = read_enumerate_fixture()
        off, pairs = o.enumerate_scan(a, b)
        assert [_partners(off, pairs, i) for i in range(a.shape[0])] == scan_lists
        off, pairs = o.enumerate_brute(a, b)
        assert [_partners(off, pairs, i) for i in range(a.shape[0])] == \
            [sorted(x) for x in scan_lists]
        return True
    except AssertionError:
        return False


def test_pins_pass_on_the_real_oracle():
    assert _pins_pass(O)


@pytest.mark.parametrize("mutant", MUTANTS)
def test_mutants_fail_pins(mutant):
    with tempfile.TemporaryDirectory() as d:
        path = oracle.build(os.path.join(d, "libmut.so"), defines=(mutant,))
        assert not _pins_pass(oracle.Oracle(oracle.load(path)))
