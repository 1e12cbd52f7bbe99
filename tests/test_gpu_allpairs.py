"""Parity of the all-pairs count matrix (the screen of Sec. "Novel genomic
relationships") with the oracle.

M[i][j] = total(A_i, B_j) from one persistent launch must equal the oracle's
Algorithm 2 total for every pair (bit-exact, uint64).
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


def oracle_matrix(a_sets, b_sets):
    built = [O.build(b) for b in b_sets]
    m = np.zeros((len(a_sets), len(b_sets)), np.uint64)
    for i, a in enumerate(a_sets):
        for j, (bs, be) in enumerate(built):
            m[i, j] = O.count_sorted(a, bs, be, threads=8, want_counts=False)[1]
    return m


@pytest.mark.parametrize("leaves", [0, 12])
def test_reduced_screen(bits, leaves):
    genome, a_sets, b_sets = synth.config5(n_sets_a=8, n_sets_b=6, hi=200_000)
    dbs = [bits.Database(dev(b), rmi_leaves_log2=leaves) for b in b_sets]
    m = bits.count_matrix(dbs, [dev(a) for a in a_sets])
    np.testing.assert_array_equal(m.cpu().numpy(), oracle_matrix(a_sets, b_sets))
    for d in dbs:
        d.free()


def test_mixed_databases_and_empty_sets(bits):
    genome, a_sets, b_sets = synth.config5(n_sets_a=5, n_sets_b=4, hi=50_000, seed=21)
    a_sets = a_sets + [np.zeros((0, 2), np.uint32), a_sets[0][:1]]
    b_sets = b_sets + [b_sets[1][:1], np.zeros((0, 2), np.uint32)]
    dbs = [bits.Database(dev(b), rmi_leaves_log2=(10 if j % 2 else 0))
           for j, b in enumerate(b_sets)]
    m = bits.count_matrix(dbs, [dev(a) for a in a_sets])
    np.testing.assert_array_equal(m.cpu().numpy(), oracle_matrix(a_sets, b_sets))
    for d in dbs:
        d.free()


def test_graph_replay_and_changed_contents(bits):
    genome, a_sets, b_sets = synth.config5(n_sets_a=4, n_sets_b=3, hi=80_000, seed=22)
    dbs = [bits.Database(dev(b)) for b in b_sets]
    da = [dev(a) for a in a_sets]
    out = torch.empty((4, 3), dtype=torch.uint64, device="cuda")
    m1 = bits.count_matrix(dbs, da, out=out).cpu().numpy().copy()
    m2 = bits.count_matrix(dbs, da, out=out).cpu().numpy().copy()
    np.testing.assert_array_equal(m1, m2)
    np.testing.assert_array_equal(m1, oracle_matrix(a_sets, b_sets))
    shifted = a_sets[2] + np.uint32(777)
    da[2].copy_(dev(shifted))
    m3 = bits.count_matrix(dbs, da, out=out).cpu().numpy()
    a_sets[2] = shifted
    np.testing.assert_array_equal(m3, oracle_matrix(a_sets, b_sets))
    for d in dbs:
        d.free()


@pytest.mark.parametrize("leaves", [16, 0])
def test_full_screen_64_by_32(bits, leaves):
    """The full 64 x 32 screen (sizes log-uniform in [1e3, 2e7], 110M queries
    counted against every database): all 2,048 entries equal the oracle's
    totals, which tests/golden/make_fullsize.py wrote from the oracle alone.
    With a learned index per database the autotuner picks each database's
    search; without one every database uses the plain tree."""
    expected = goldens.read_allpairs_fullsize()
    genome, a_sets, b_sets = synth.config5()
    dbs = [bits.Database(dev(b), rmi_leaves_log2=leaves) for b in b_sets]
    da = [dev(a) for a in a_sets]
    m = bits.count_matrix(dbs, da).cpu().numpy()
    np.testing.assert_array_equal(m, expected)
    for d in dbs:
        d.free()


# ---- bits_count_matrix_db: both sides given as databases ---------------------

def test_matrix_db_reduced_and_mirrored(bits):
    """Every pair counted from its smaller side's sorted keys in the larger
    side's tree equals the oracle's total (sizes up to 2e5, so both
    directions occur), and swapping the two lists transposes the matrix."""
    genome, a_sets, b_sets = synth.config5(n_sets_a=8, n_sets_b=6, hi=200_000, seed=23)
    a_dbs = [bits.Database(dev(a)) for a in a_sets]
    b_dbs = [bits.Database(dev(b), rmi_leaves_log2=(12 if j % 2 else 0))
             for j, b in enumerate(b_sets)]
    m = bits.count_matrix_db(a_dbs, b_dbs).cpu().numpy()
    np.testing.assert_array_equal(m, oracle_matrix(a_sets, b_sets))
    mt = bits.count_matrix_db(b_dbs, a_dbs).cpu().numpy()
    np.testing.assert_array_equal(mt, m.T)
    for d in a_dbs + b_dbs:
        d.free()


def test_matrix_db_ties_tiny_and_empty(bits):
    """Equal sizes (the A side counts), sets of one interval, empty
    databases on either side, and a set against itself."""
    genome, a_sets, b_sets = synth.config5(n_sets_a=3, n_sets_b=3, hi=30_000, seed=24)
    a_sets = a_sets + [b_sets[0].copy(), a_sets[0][:1], np.zeros((0, 2), np.uint32)]
    b_sets = b_sets + [a_sets[1].copy(), np.zeros((0, 2), np.uint32)]
    a_dbs = [bits.Database(dev(a)) for a in a_sets]
    b_dbs = [bits.Database(dev(b)) for b in b_sets]
    out = torch.empty((len(a_sets), len(b_sets)), dtype=torch.uint64, device="cuda")
    m1 = bits.count_matrix_db(a_dbs, b_dbs, out=out).cpu().numpy().copy()
    m2 = bits.count_matrix_db(a_dbs, b_dbs, out=out).cpu().numpy()   # graph replay
    np.testing.assert_array_equal(m1, oracle_matrix(a_sets, b_sets))
    np.testing.assert_array_equal(m2, m1)
    for d in a_dbs + b_dbs:
        d.free()


def test_matrix_db_full_screen_64_by_32(bits):
    """The full 64 x 32 screen with the 64 query sets built as databases:
    all 2,048 entries equal the oracle's stored totals."""
    expected = goldens.read_allpairs_fullsize()
    genome, a_sets, b_sets = synth.config5()
    a_dbs = [bits.Database(dev(a)) for a in a_sets]
    b_dbs = [bits.Database(dev(b)) for b in b_sets]
    m = bits.count_matrix_db(a_dbs, b_dbs).cpu().numpy()
    np.testing.assert_array_equal(m, expected)
    for d in a_dbs + b_dbs:
        d.free()
