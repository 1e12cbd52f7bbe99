"""Parity of the merge-path form of bits_count with the oracle.

The queries' end keys and start+1 keys are sorted with their indices and
co-ranked against B_S and B_E by merge path; per-query counts and totals
must equal the oracle's Algorithm 2 bit for bit, and equal the plain search
on the same queries.
"""
import numpy as np
import pytest
import torch

import bits_synth as synth
import oracle

pytestmark = pytest.mark.gpu

O = oracle.get()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32)).cuda()


@pytest.fixture(scope="module")
def bits():
    import paper_1208_3407_b300 as bits
    return bits


def mp_count(bits, a, b, counts=True):
    db = bits.Database(dev(b))
    c, t = db.count(dev(a), counts=counts, method=bits.METHOD_MERGEPATH)
    out = (c.cpu().numpy() if c is not None else None), int(t.cpu().numpy()[0])
    db.free()
    return out


@pytest.mark.parametrize("n_a,n_b", [(1, 1), (2047, 1), (2049, 3000), (300_001, 299_999),
                                     (50_000, 2_000_000), (1_000_003, 20_000), (8192 * 3 + 1, 8192)])
def test_sizes(bits, n_a, n_b):
    _, a, b = synth.config2(n_a=n_a, n_b=n_b, n_hot=max(1, n_b // 10))
    c, t = mp_count(bits, a, b)
    oc, ot = O.count(a, b, threads=8)
    np.testing.assert_array_equal(c, oc)
    assert t == ot
    _, t2 = mp_count(bits, a, b, counts=False)
    assert t2 == ot


@pytest.mark.parametrize("seed", range(10))
def test_tiny_random_with_ties(bits, seed):
    rng = np.random.default_rng(100 + seed)
    a, b = synth.tiny_random(seed, int(rng.integers(1, 5000)), int(rng.integers(1, 5000)),
                             coord_max=int(rng.integers(4, 300)), max_len=int(rng.integers(1, 30)))
    c, t = mp_count(bits, a, b)
    bc, bt = O.count_brute(a, b)
    np.testing.assert_array_equal(c, bc)
    assert t == bt


def test_golden_and_extremes(bits):
    from goldens import read_count_fixture
    for name in ("containment.txt", "duplicates.txt"):
        a, b, exp, total = read_count_fixture(name)
        c, t = mp_count(bits, a, b)
        np.testing.assert_array_equal(c, exp)
        assert t == total
    top = 2**32 - 1
    b = np.array([[top - 5, top], [0, 1], [top - 1, top]], np.uint32)
    a = np.array([[top - 1, top - 1], [top - 2, top], [top, top], [0, 0], [0, top]], np.uint32)
    c, t = mp_count(bits, a, b)
    np.testing.assert_array_equal(c, O.count_brute(a, b)[0])
    c, t = mp_count(bits, a, np.zeros((0, 2), np.uint32))
    assert t == 0 and (c == 0).all()


def test_inverted_queries_match_plain_search(bits):
    _, a, b = synth.config2(n_a=20_000, n_b=100_000, n_hot=1000)
    bad = a.copy()
    bad[::97, 0], bad[::97, 1] = a[::97, 1] + 5, a[::97, 0]
    db = bits.Database(dev(b))
    for counts in (True, False):
        outs = []
        for m in (bits.METHOD_SEARCH, bits.METHOD_MERGEPATH):
            with pytest.raises(bits.BitsError):
                db.count(dev(bad), counts=counts, method=m)
            c, t = db.count(dev(bad), counts=counts, method=m, check=False)
            outs.append(((c.cpu().numpy() if c is not None else None), int(t.cpu().numpy()[0])))
            with pytest.raises(bits.BitsError):
                db.check()
        if counts:
            np.testing.assert_array_equal(outs[0][0], outs[1][0])
        assert outs[0][1] == outs[1][1]
    good = np.ones(a.shape[0], bool)
    good[::97] = False
    assert outs[1][1] == O.count(a[good], b)[1]
    db.free()


def test_config4_full_size_mergepath_vs_plain(bits):
    a, b = synth.config4()
    db = bits.Database(dev(b))
    da = dev(a)
    c_m, t_m = db.count(da, method=bits.METHOD_MERGEPATH)
    c_p, t_p = db.count(da, method=bits.METHOD_SEARCH)
    assert torch.equal(c_m.view(torch.int32), c_p.view(torch.int32))
    _, t_tot = db.count(da, counts=False, method=bits.METHOD_MERGEPATH)
    assert int(t_m.cpu().numpy()[0]) == int(t_p.cpu().numpy()[0]) == int(t_tot.cpu().numpy()[0])
    db.free()
