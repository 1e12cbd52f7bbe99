"""Parity of the Monte-Carlo summary (Sec. "Monte Carlo Simulations" tallies,
Fig. 3 score) and of the Monte-Carlo screen over query sets x databases (Sec.
"Novel genomic relationships") with the oracle.

Integer fields and p-values must match bit for bit.  The enrichment score is
log2 of one IEEE division: the division is exact on both sides, and CUDA's
double log2 is within 1 ulp of the true value, as is glibc's, so the two
may differ by at most 2 ulp.
"""
import math

import numpy as np
import pytest
import torch

import bits_synth as synth
import oracle
from goldens import read_mc_summary_fixture

pytestmark = pytest.mark.gpu

O = oracle.get()
INTS = ("observed", "k_ge", "k_le", "median_lo", "median_hi")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32)).cuda()


def dev64(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint64)).cuda()


@pytest.fixture(scope="module")
def bits():
    import paper_1208_3407_b300 as bits
    return bits


def assert_stat(got: dict, exp: dict, where=""):
    for k in INTS:
        assert got[k] == exp[k], (where, k, got[k], exp[k])
    assert got["p_enrich"] == exp["p_enrich"], where
    assert got["p_deplete"] == exp["p_deplete"], where
    g, e = got["log2_enrichment"], exp["log2_enrichment"]
    if math.isnan(e) or math.isinf(e):
        assert (math.isnan(g) and math.isnan(e)) or g == e, (where, g, e)
    else:
        assert abs(g - e) <= 2 * np.spacing(abs(e)) + (0.0 if e else 0.0), (where, g, e)


# ----------------------------------------------------------------- summary

def test_summary_golden(bits):
    for obs, totals, exp in read_mc_summary_fixture():
        st = bits.mc_summary(dev64(totals).view(1, -1), dev64([obs])).to_dicts()[0]
        assert_stat(st, O.mc_summary(totals, obs), where=(obs, list(totals)))
        for k in ("k_ge", "k_le", "median_lo", "median_hi"):
            assert st[k] == exp[k]


def _batch(rng, kind, n_tests, n):
    if kind == "clustered":            # shuffled totals around 1e9, a few thousand apart
        t = 1_000_000_000 + rng.integers(-3000, 3000, size=(n_tests, n))
        o = 1_000_000_000 + rng.integers(-4000, 4000, size=n_tests)
    elif kind == "wide":               # every byte of the 63-bit range in play
        t = rng.integers(0, 2**62, size=(n_tests, n)) * 2 + rng.integers(0, 2, size=(n_tests, n))
        o = rng.integers(0, 2**62, size=n_tests)
    elif kind == "ties":
        t = rng.integers(5, 8, size=(n_tests, n))
        o = rng.integers(4, 9, size=n_tests)
    else:                              # zeros: many empty shuffles
        t = rng.integers(0, 2, size=(n_tests, n)) * rng.integers(0, 3, size=(n_tests, n))
        o = rng.integers(0, 2, size=n_tests)
    return t.astype(np.uint64), o.astype(np.uint64)


@pytest.mark.parametrize("kind", ["clustered", "wide", "ties", "zeros"])
@pytest.mark.parametrize("n", [1, 2, 3, 255, 256, 1000, 10_000, 10_001])
def test_summary_random(bits, kind, n):
    rng = np.random.default_rng(n * 7 + len(kind))
    n_tests = 37 if n <= 1000 else 9
    t, o = _batch(rng, kind, n_tests, n)
    got = bits.mc_summary(dev64(t), dev64(o)).to_dicts()
    for i in range(n_tests):
        assert_stat(got[i], O.mc_summary(t[i], int(o[i])), where=(kind, n, i))


def test_summary_zero_shuffles_and_overflow(bits):
    st = bits.mc_summary(torch.empty((3, 0), dtype=torch.uint64, device="cuda"),
                         dev64([0, 5, 9])).to_dicts()
    for i, obs in enumerate((0, 5, 9)):
        assert st[i]["k_ge"] == 0 and st[i]["k_le"] == 0
        assert st[i]["median_lo"] == 0 and st[i]["median_hi"] == 0
        assert st[i]["p_enrich"] == 1.0 and st[i]["p_deplete"] == 1.0
    # 2 * observed past 64 bits: the score is NaN, the tallies stay exact.
    big = np.array([[2**63, 2**63 + 5, 3]], np.uint64)
    st = bits.mc_summary(dev64(big), dev64([2**63 + 1])).to_dicts()[0]
    assert math.isnan(st["log2_enrichment"])
    assert st["k_ge"] == 1 and st["k_le"] == 2 and st["median_lo"] == 2**63


def test_summary_views(bits):
    t = dev64(np.arange(12, dtype=np.uint64).reshape(2, 2, 3))
    s = bits.mc_summary(t, dev64([[1, 2], [8, 100]]))
    assert s.k_ge.shape == (2, 2) and s.p_enrich.dtype == torch.float64
    assert s.median_lo.cpu().tolist() == [[1, 4], [7, 10]]


# ----------------------------------------------------------------- screen

def _screen_inputs(sizes_a, sizes_b, seed=0):
    genome = synth.make_genome(n_contigs=6, lo=200_000, hi=900_000, seed=seed + 1)
    a_sets = [synth.config5_set(2 * i, n, genome, seed=seed + 40) for i, n in enumerate(sizes_a)]
    b_sets = [synth.config5_set(2 * i + 1, n, genome, seed=seed + 41)
              for i, n in enumerate(sizes_b)]
    return genome, a_sets, b_sets


def _oracle_screen(genome, a_sets, b_sets, seed, s0, s1):
    co, cl = synth.mc_contig_table(genome)
    built = [O.build(b) for b in b_sets]
    obs = np.zeros((len(a_sets), len(b_sets)), np.uint64)
    tot = np.zeros((len(a_sets), len(b_sets), s1 - s0), np.uint64)
    for i, a in enumerate(a_sets):
        for j, (bs, be) in enumerate(built):
            t, o, _, _ = O.mc(a, co, cl, bs, be, seed=seed, s_begin=s0, s_end=s1, threads=8,
                              set_index=i)
            tot[i, j] = t
            obs[i, j] = o
    return obs, tot


def _gpu_screen(bits, genome, a_sets, b_sets, seed, s0, s1, stats=True):
    co, cl = synth.mc_contig_table(genome)
    dbs = [bits.Database(dev(b)) for b in b_sets]
    obs, tot, st = bits.mc_matrix(dbs, [dev(a) for a in a_sets], dev(co), dev(cl), seed=seed,
                                  shuffle_begin=s0, shuffle_end=s1, stats=stats)
    torch.cuda.synchronize()
    for d in dbs:
        d.check()
    out = obs.cpu().numpy().copy(), tot.cpu().numpy().copy(), (st.to_dicts() if st else None)
    for d in dbs:
        d.free()
    return out


@pytest.mark.parametrize("sizes_a,sizes_b,n_sh", [
    ([1, 500, 2500], [1, 3000], 40),           # ragged chunks, a one-interval set and database
    ([1025, 0, 64, 3000, 7], [200, 50_000, 9], 257),   # an empty set, > one shuffle block
    ([4000], [20_000], 513),
])
def test_screen_parity(bits, sizes_a, sizes_b, n_sh):
    genome, a_sets, b_sets = _screen_inputs(sizes_a, sizes_b, seed=len(sizes_a))
    obs, tot, st = _gpu_screen(bits, genome, a_sets, b_sets, 99, 3, 3 + n_sh)
    oobs, otot = _oracle_screen(genome, a_sets, b_sets, 99, 3, 3 + n_sh)
    np.testing.assert_array_equal(obs, oobs)
    np.testing.assert_array_equal(tot, otot)
    for i in range(len(a_sets)):
        for j in range(len(b_sets)):
            assert_stat(st[i * len(b_sets) + j], O.mc_summary(otot[i, j], int(oobs[i, j])),
                        where=(i, j))


def test_screen_set0_is_single_test_and_resumable(bits):
    genome, a_sets, b_sets = _screen_inputs([800, 1500], [5000, 700], seed=5)
    co, cl = synth.mc_contig_table(genome)
    _, tot, _ = _gpu_screen(bits, genome, a_sets, b_sets, 7, 0, 60, stats=False)
    for j, b in enumerate(b_sets):
        db = bits.Database(dev(b))
        t, *_ = db.mc(dev(a_sets[0]), dev(co), dev(cl), seed=7, shuffle_end=60,
                      method=bits.METHOD_SEARCH)
        np.testing.assert_array_equal(t.cpu().numpy(), tot[0, j])
        db.free()
    _, t_lo, _ = _gpu_screen(bits, genome, a_sets, b_sets, 7, 0, 25, stats=False)
    _, t_hi, _ = _gpu_screen(bits, genome, a_sets, b_sets, 7, 25, 60, stats=False)
    np.testing.assert_array_equal(np.concatenate([t_lo, t_hi], axis=2), tot)
    # Sets differ only through their stream: the same intervals as set 0 and 1
    # give different shuffled totals.
    _, tot2, _ = _gpu_screen(bits, genome, [a_sets[0], a_sets[0]], b_sets, 7, 0, 60, stats=False)
    np.testing.assert_array_equal(tot2[0], tot[0])
    assert not np.array_equal(tot2[1], tot2[0])


def test_screen_replay_and_invalid_interval(bits):
    genome, a_sets, b_sets = _screen_inputs([300, 900], [4000, 100], seed=8)
    co, cl = synth.mc_contig_table(genome)
    dbs = [bits.Database(dev(b)) for b in b_sets]
    a_dev = [dev(a) for a in a_sets]
    args = dict(seed=3, shuffle_end=20)
    o1, t1, _ = bits.mc_matrix(dbs, a_dev, dev(co), dev(cl), **args)
    t1 = t1.cpu().numpy().copy()
    # Replay of the cached graph with the same buffers gives the same totals.
    obs2, tot2, _ = bits.mc_matrix(dbs, a_dev, dev(co), dev(cl), **args)
    np.testing.assert_array_equal(tot2.cpu().numpy(), t1)
    # An interval crossing its contig's end flags every database it met.
    bad = a_sets[1].copy()
    last = int(genome.offsets[-1] + genome.lengths[-1])
    bad[0] = (last - 5, last + 5)
    bits.mc_matrix(dbs, [a_dev[0], dev(bad)], dev(co), dev(cl), **args)
    torch.cuda.synchronize()
    for d in dbs:
        with pytest.raises(bits.BitsError):
            d.check()
        d.free()


def test_screen_larger_sampled(bits):
    # 8 query sets x 4 databases, sizes log-uniform up to 1e5, 16 shuffles.
    sizes_a = [100_000, 3_000, 45_000, 800, 12_000, 60_000, 1_500, 25_000]
    sizes_b = [100_000, 10_000, 400_000, 2_000]
    genome, a_sets, b_sets = _screen_inputs(sizes_a, sizes_b, seed=12)
    obs, tot, st = _gpu_screen(bits, genome, a_sets, b_sets, 1234, 0, 16)
    co, cl = synth.mc_contig_table(genome)
    for i, j in ((0, 2), (3, 1), (5, 0), (7, 3)):
        bs, be = O.build(b_sets[j])
        t, o, _, _ = O.mc(a_sets[i], co, cl, bs, be, seed=1234, s_begin=0, s_end=16, threads=8,
                          set_index=i)
        np.testing.assert_array_equal(tot[i, j], t)
        assert obs[i, j] == o
        assert_stat(st[i * 4 + j], O.mc_summary(t, o), where=(i, j))


def test_screen_by_databases(bits):
    """Sets far larger than many small databases: the screen builds each
    shuffle's placed sets as databases and counts every pair from its
    smaller side.  Every total, observed count and summary equals the
    oracle's; shuffle ranges split and rejoin; with one empty query interval
    (which no database may hold) the same screen runs in the persistent
    kernel and gives the same totals."""
    sizes_a = [400_000, 350_000, 300_000]
    sizes_b = [2_000, 1_500, 2_500, 1_000, 3_000, 2_200, 900, 1_800, 2_600, 1_200, 2_000, 1_700]
    genome, a_sets, b_sets = _screen_inputs(sizes_a, sizes_b, seed=31)
    obs, tot, st = _gpu_screen(bits, genome, a_sets, b_sets, 4242, 0, 6)
    oobs, otot = _oracle_screen(genome, a_sets, b_sets, 4242, 0, 6)
    np.testing.assert_array_equal(obs, oobs)
    np.testing.assert_array_equal(tot, otot)
    for i in range(len(a_sets)):
        for j in range(len(b_sets)):
            assert_stat(st[i * len(b_sets) + j], O.mc_summary(otot[i, j], int(oobs[i, j])),
                        where=(i, j))
    _, t_lo, _ = _gpu_screen(bits, genome, a_sets, b_sets, 4242, 0, 2, stats=False)
    _, t_hi, _ = _gpu_screen(bits, genome, a_sets, b_sets, 4242, 2, 6, stats=False)
    np.testing.assert_array_equal(np.concatenate([t_lo, t_hi], axis=2), tot)
    empty = [a.copy() for a in a_sets]
    empty[1][7, 1] = empty[1][7, 0]
    obs_e, tot_e, _ = _gpu_screen(bits, genome, empty, b_sets, 4242, 0, 6, stats=False)
    oobs_e, otot_e = _oracle_screen(genome, empty, b_sets, 4242, 0, 6)
    np.testing.assert_array_equal(tot_e, otot_e)
    np.testing.assert_array_equal(obs_e, oobs_e)
