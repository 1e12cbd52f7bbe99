"""The learned-index form gives exactly the plain search's counts.

The learned index (a linear root over 2^L linear leaves with per-leaf error
bounds, fitted on the device) is not in the paper; it replaces the first
steps of each BSearch of Algorithm 1.  Its counts must equal the oracle's and
the plain search's bit for bit, including when its error bounds are wrong.
"""
import os

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


def both_forms(bits, a, b, leaves_log2, **kw):
    db = bits.Database(dev(b), rmi_leaves_log2=leaves_log2, **kw)
    da = dev(a)
    c_rmi, t_rmi = db.count(da, method=bits.METHOD_RMI)
    c_pl, t_pl = db.count(da, method=bits.METHOD_SEARCH)
    out = (c_rmi.cpu().numpy(), int(t_rmi.cpu().numpy()[0]),
           c_pl.cpu().numpy(), int(t_pl.cpu().numpy()[0]))
    return db, out


@pytest.mark.parametrize("leaves_log2", [1, 4, 10, 16])
def test_config2_reduced(bits, leaves_log2):
    _, a, b = synth.config2(n_a=50_001, n_b=1_000_003, n_hot=10_000)
    db, (cr, tr, cp, tp) = both_forms(bits, a, b, leaves_log2)
    oc, ot = O.count(a, b, threads=8)
    np.testing.assert_array_equal(cr, oc)
    np.testing.assert_array_equal(cp, oc)
    assert tr == tp == ot
    db.free()


@pytest.mark.parametrize("seed", range(12))
def test_tiny_and_degenerate(bits, seed):
    rng = np.random.default_rng(seed)
    na, nb = int(rng.integers(1, 500)), int(rng.integers(1, 3000))
    a, b = synth.tiny_random(seed, na, nb, coord_max=int(rng.integers(8, 5000)),
                             max_len=int(rng.integers(1, 60)))
    db, (cr, tr, cp, tp) = both_forms(bits, a, b, int(rng.integers(1, 14)),
                                      top_tree_log2=int(rng.integers(2, 10)))
    bc, bt = O.count_brute(a, b)
    np.testing.assert_array_equal(cr, bc)
    assert tr == bt
    db.free()


def test_all_equal_keys_and_empty(bits):
    a, _ = synth.config1(n_a=2000)
    same = np.tile(np.array([[500_000, 500_100]], np.uint32), (50_000, 1))
    db, (cr, tr, cp, tp) = both_forms(bits, a, same, 16)
    oc, ot = O.count(a, same)
    np.testing.assert_array_equal(cr, oc)
    db.free()
    db, (cr, tr, cp, tp) = both_forms(bits, a, np.zeros((0, 2), np.uint32), 8)
    assert tr == 0 and (cr == 0).all()
    db.free()


def test_config4_reduced_skewed_mixture(bits):
    a, b = synth.config4(n_a=200_000, n_b=2_000_000)
    db, (cr, tr, cp, tp) = both_forms(bits, a, b, 16)
    oc, ot = O.count(a, b, threads=8)
    np.testing.assert_array_equal(cr, oc)
    np.testing.assert_array_equal(cp, oc)
    assert tr == ot
    db.free()


def test_wrong_error_bounds_still_exact(bits):
    _, a, b = synth.config2(n_a=30_000, n_b=400_000, n_hot=3000)
    db = bits.Database(dev(b), rmi_leaves_log2=12)
    oc, ot = O.count(a, b)
    rng = np.random.default_rng(5)
    for which in (0, 1):
        leaves, _, _ = db.rmi(which)
        nl = leaves.shape[0]
        # Collapse the bounds of every third leaf to [0, 0] and push a few
        # windows off the slice entirely.
        idx = torch.arange(0, nl, 3, device="cuda")
        leaves[idx, 4] = 0
        leaves[idx, 5] = 0
        far = torch.tensor(rng.choice(nl, size=min(50, nl), replace=False), device="cuda")
        leaves[far, 4] = 1000
        leaves[far, 5] = 2000
    torch.cuda.synchronize()
    c, t = db.count(dev(a), method=bits.METHOD_RMI)
    np.testing.assert_array_equal(c.cpu().numpy(), oc)
    assert int(t.cpu().numpy()[0]) == ot
    db.free()


def test_leaf_table_is_consistent(bits):
    _, _, b = synth.config3(n_a=1, n_b=300_000, n_hot=3000)
    db = bits.Database(dev(b), rmi_leaves_log2=10)
    for which in (0, 1):
        leaves, ra, rb = db.rmi(which)
        t = leaves.cpu().numpy()
        lo, hi = t[:, 1].astype(np.int64), t[:, 6].astype(np.int64)
        assert lo[0] == 0 and hi[-1] == b.shape[0]
        np.testing.assert_array_equal(hi[:-1], lo[1:])          # slices tile [0, n)
        assert (t[:, 4] <= 0).all() and (t[:, 5] >= 0).all()    # window holds offset 0
        assert ra >= 0.0
    db.free()


def test_mc_learned_index_equals_plain_and_oracle(bits):
    genome, a, b = synth.config3(n_a=3000, n_b=50_000, n_hot=5000)
    co, cl = synth.mc_contig_table(genome)
    db = bits.Database(dev(b), rmi_leaves_log2=12)
    t_r, o_r, k_r, p_r = db.mc(dev(a), dev(co), dev(cl), seed=7, shuffle_end=300,
                               method=bits.METHOD_RMI)
    t_r = t_r.cpu().numpy().copy()
    t_p, o_p, k_p, p_p = db.mc(dev(a), dev(co), dev(cl), seed=7, shuffle_end=300,
                               method=bits.METHOD_SEARCH)
    np.testing.assert_array_equal(t_r, t_p.cpu().numpy())
    bs, be = O.build(b)
    ot, oobs, ok, op = O.mc(a, co, cl, bs, be, seed=7, s_begin=0, s_end=300, threads=8)
    np.testing.assert_array_equal(t_r, ot)
    assert (o_r, k_r, p_r) == (oobs, ok, op) == (o_p, k_p, p_p)
    db.free()


def test_config4_full_size_learned_vs_plain(bits):
    """100M queries vs 100M intervals, 2^16 leaves: both forms bit-exact with
    each other and with the oracle's count of every query (std::sort and
    std::lower_bound on the host, all cores); 64 sampled queries are also
    recomputed by brute force."""
    a, b = synth.config4()
    db = bits.Database(dev(b), rmi_leaves_log2=16)
    da = dev(a)
    c_r, t_r = db.count(da, method=bits.METHOD_RMI)
    c_p, t_p = db.count(da, method=bits.METHOD_SEARCH)
    assert torch.equal(c_r.view(torch.int32), c_p.view(torch.int32))
    total = int(c_r.view(torch.int32).to(torch.int64).sum().item())
    assert int(t_r.cpu().numpy()[0]) == int(t_p.cpu().numpy()[0]) == total
    bs, be = db.sorted_arrays()
    for x in (bs, be):
        x64 = x.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        assert bool((x64[1:] >= x64[:-1]).all())
        del x64
    got = c_r.cpu().numpy()
    obs, obe = O.build(b)
    oc_all, ot_all = O.count_sorted(a, obs, obe, threads=os.cpu_count() or 1)
    np.testing.assert_array_equal(got, oc_all)
    assert ot_all == total
    idx = np.random.default_rng(1).choice(a.shape[0], size=64, replace=False)
    oc, _ = O.count_brute(a[idx], b)
    np.testing.assert_array_equal(got[idx], oc)
    db.free()
