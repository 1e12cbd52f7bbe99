"""Parity of the Monte-Carlo significance test (Sec. "Monte Carlo Simulations") with the CPU oracle.

Per-shuffle totals, the observed total, k_ge and the p-value must match the
oracle bit-exactly on the same seeded inputs and the same Philox counters.
"""
import numpy as np
import pytest
import torch

import bits_synth as synth
import goldens
import oracle

pytestmark = pytest.mark.gpu

O = oracle.get()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32)).cuda()


@pytest.fixture(scope="module")
def bits():
    import paper_1208_3407_b300 as bits
    return bits


def run_both(bits, genome, a, b, seed, s0, s1, method=None, db=None):
    import paper_1208_3407_b300 as bm
    method = bm.METHOD_SEARCH if method is None else method
    co, cl = synth.mc_contig_table(genome)
    own = db is None
    if own:
        db = bits.Database(dev(b))
    totals, obs, k, p = db.mc(dev(a), dev(co), dev(cl), seed=seed, shuffle_begin=s0,
                              shuffle_end=s1, method=method)
    t = totals.cpu().numpy().copy()
    if own:
        db.free()
    bs, be = O.build(b)
    ot, oobs, ok, op = O.mc(a, co, cl, bs, be, seed=seed, s_begin=s0, s_end=s1, threads=8)
    return (t, obs, k, p), (ot, oobs, ok, op)


@pytest.mark.parametrize("n_a,n_b,n_sh", [(1, 10, 1), (2000, 20_000, 300), (1025, 5000, 257),
                                          (3000, 1, 64), (4099, 100_000, 513)])
def test_small_cases(bits, n_a, n_b, n_sh):
    genome, a, b = synth.config3(n_a=n_a, n_b=n_b, n_hot=max(1, n_b // 5))
    (t, obs, k, p), (ot, oobs, ok, op) = run_both(bits, genome, a, b, 7, 0, n_sh)
    np.testing.assert_array_equal(t, ot)
    assert (obs, k, p) == (oobs, ok, op)


def test_resumable_ranges_and_seed(bits):
    genome, a, b = synth.config3(n_a=1500, n_b=30_000, n_hot=3000)
    (t, *_), (ot, *_) = run_both(bits, genome, a, b, 2**40 + 12345, 100, 400)
    np.testing.assert_array_equal(t, ot)
    (t0, *_), _ = run_both(bits, genome, a, b, 2**40 + 12345, 0, 400)
    np.testing.assert_array_equal(t0[100:], t)


def test_graph_replay_reads_current_inputs(bits):
    genome, a, b = synth.config3(n_a=2000, n_b=40_000, n_hot=4000)
    co, cl = synth.mc_contig_table(genome)
    db = bits.Database(dev(b))
    da, dco, dcl = dev(a), dev(co), dev(cl)
    totals = torch.empty(200, dtype=torch.uint64, device="cuda")
    r1 = db.mc(da, dco, dcl, seed=3, shuffle_end=200, totals=totals, method=bits.METHOD_SEARCH)
    t1 = totals.cpu().numpy().copy()
    r2 = db.mc(da, dco, dcl, seed=3, shuffle_end=200, totals=totals, method=bits.METHOD_SEARCH)
    np.testing.assert_array_equal(totals.cpu().numpy(), t1)
    assert r1[1:] == r2[1:]
    # Same pointers, new contents: the replayed graph must see them.
    _, a2, _ = synth.config3(n_a=2000, n_b=10, seed_a=99)
    da.copy_(dev(a2))
    r3 = db.mc(da, dco, dcl, seed=3, shuffle_end=200, totals=totals, method=bits.METHOD_SEARCH)
    bs, be = O.build(b)
    ot, oobs, ok, op = O.mc(a2, co, cl, bs, be, seed=3, s_begin=0, s_end=200, threads=8)
    np.testing.assert_array_equal(totals.cpu().numpy(), ot)
    assert r3[1:] == (oobs, ok, op)
    db.free()


def test_degenerate_contig_is_deterministic(bits):
    genome = synth.Genome(np.array([0, 100, 300], np.uint32), np.array([100, 200, 50], np.uint32), 350)
    a = np.array([[0, 100], [100, 300], [300, 350]], np.uint32)
    b = np.array([[50, 60], [99, 101], [299, 301], [340, 345], [0, 400]], np.uint32)
    (t, obs, k, p), (ot, oobs, ok, op) = run_both(bits, genome, a, b, 5, 0, 16)
    np.testing.assert_array_equal(t, ot)
    assert (t == obs).all() and k == 16 and p == 1.0


def test_empty_and_zero_shuffles(bits):
    genome, a, b = synth.config3(n_a=100, n_b=1000, n_hot=10)
    (t, obs, k, p), (ot, oobs, ok, op) = run_both(bits, genome, a, b, 1, 5, 5)
    assert t.shape == (0,) and (obs, k, p) == (oobs, ok, op) and p == 1.0
    (t, obs, k, p), (ot, oobs, ok, op) = run_both(bits, genome, a[:0], b, 1, 0, 10)
    assert (t == 0).all() and obs == 0 and k == 10 and p == 1.0


def test_interval_crossing_contig_is_rejected(bits):
    genome, a, b = synth.config3(n_a=100, n_b=1000, n_hot=10)
    co, cl = synth.mc_contig_table(genome)
    bad = a.copy()
    bad[5] = [int(co[1]) - 10, int(co[1]) + 10]
    db = bits.Database(dev(b))
    with pytest.raises(bits.BitsError) as e:
        db.mc(dev(bad), dev(co), dev(cl), seed=1, shuffle_end=8, method=bits.METHOD_SEARCH)
    assert e.value.status == 1
    db.free()


@pytest.mark.parametrize("method", ["search", "rmi"])
def test_config3_full_size_every_shuffle(bits, method):
    """Table 1's 1e5 x 1e4 corner at full size: 10,000 shuffles of 100,000
    intervals against 1,000,000 in one launch.  Every per-shuffle total, the
    observed total, k_ge and the p-value equal the oracle's, which
    tests/golden/make_fullsize.py wrote from the oracle alone (the full run
    takes about a minute on eight host cores)."""
    gobs, gk, (pnum, pden), gtot = goldens.read_mc_fullsize()
    genome, a, b = synth.config3()
    co, cl = synth.mc_contig_table(genome)
    db = bits.Database(dev(b), rmi_leaves_log2=16 if method == "rmi" else 0)
    m = bits.METHOD_RMI if method == "rmi" else bits.METHOD_SEARCH
    totals, obs, k, p = db.mc(dev(a), dev(co), dev(cl), seed=7, shuffle_end=10_000, method=m)
    t = totals.cpu().numpy()
    db.free()
    np.testing.assert_array_equal(t, gtot)
    assert (obs, k) == (gobs, gk)
    assert p == pnum / pden
