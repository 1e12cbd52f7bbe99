"""Parity of the CUDA enumeration (the enumeration problem of Sec. "Interval
Set Intersection problem", the count-terminated scan of Sec. "BITS Algorithm")
with the CPU oracle.

Offsets and pairs must equal the oracle's scan bit for bit, order included
(descending start, equal starts by descending index), and each query's
partners must be the set the definition gives.
"""
import numpy as np
import pytest
import torch

import bits_synth as synth
import oracle
from goldens import read_enumerate_fixture

pytestmark = pytest.mark.gpu

O = oracle.get()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32)).cuda()


@pytest.fixture(scope="module")
def bits():
    import paper_1208_3407_b300 as bits
    return bits


def gpu_enum(bits, a, b):
    db = bits.Database(dev(b), enumerate=True)
    off, pairs = db.enumerate(dev(a))
    out = off.cpu().numpy().copy(), pairs.cpu().numpy().copy()
    db.free()
    return out


def assert_parity(bits, a, b, check_sets=True):
    off, pairs = gpu_enum(bits, a, b)
    eoff, epairs = O.enumerate_scan(a, b)
    np.testing.assert_array_equal(off, eoff)
    np.testing.assert_array_equal(pairs, epairs)
    if check_sets:
        boff, bpairs = O.enumerate_brute(a, b)
        np.testing.assert_array_equal(off, boff)
        for i in range(a.shape[0]):
            lo, hi = int(off[i]), int(off[i + 1])
            assert sorted(pairs[lo:hi, 1].tolist()) == bpairs[lo:hi, 1].tolist()


def test_golden(bits):
    a, b, exp, total, scan_lists = read_enumerate_fixture()
    off, pairs = gpu_enum(bits, a, b)
    assert int(off[-1]) == total
    for i, want in enumerate(scan_lists):
        lo, hi = int(off[i]), int(off[i + 1])
        assert pairs[lo:hi, 1].tolist() == want
        assert (pairs[lo:hi, 0] == i).all()


@pytest.mark.parametrize("seed", range(12))
def test_tiny_random(bits, seed):
    a, b = synth.tiny_random(seed, n_a=50 + 37 * seed, n_b=70 + 53 * seed, coord_max=300,
                             max_len=60)
    assert_parity(bits, a, b)


def test_nested_containment(bits):
    # Every query lies under the outermost intervals and right of many
    # contained ones: long scans, counts from the nested closed form.
    m = 3000
    b = synth.nested(m)
    x = np.arange(0, 2 * m + 5, 7)
    a = np.stack([x, x + 1], 1).astype(np.uint32)
    assert_parity(bits, a, b, check_sets=False)


@pytest.mark.parametrize("n_a,n_b", [(1, 1), (33, 5000), (20_000, 200_000), (65_537, 1_000)])
def test_config_shapes(bits, n_a, n_b):
    _, a, b = synth.config2(n_a=n_a, n_b=n_b, n_hot=max(1, n_b // 100))
    assert_parity(bits, a, b, check_sets=n_a * n_b <= 1e8)


def test_full_size_exome_vs_reads(bits):
    # 200,000 queries against 20,000,000 reads: every pair, in order.
    _, a, b = synth.config2()
    off, pairs = gpu_enum(bits, a, b)
    eoff, epairs = O.enumerate_scan(a, b)
    np.testing.assert_array_equal(off, eoff)
    np.testing.assert_array_equal(pairs, epairs)
    counts, total = O.count(a, b, threads=8)
    assert int(off[-1]) == total
    np.testing.assert_array_equal(np.diff(off.astype(np.int64)), counts)


def test_empty_inputs(bits):
    b = np.array([[5, 9]], np.uint32)
    off, pairs = gpu_enum(bits, np.zeros((0, 2), np.uint32), b)
    assert off.tolist() == [0] and pairs.shape == (0, 2)
    a = np.array([[0, 3], [4, 6]], np.uint32)
    off, pairs = gpu_enum(bits, a, np.zeros((0, 2), np.uint32))
    assert off.tolist() == [0, 0, 0] and pairs.shape == (0, 2)


def test_errors(bits):
    b = dev(np.array([[5, 9], [1, 20]], np.uint32))
    a = dev(np.array([[6, 7], [0, 3]], np.uint32))
    db = bits.Database(b)                     # built without the enumeration arrays
    with pytest.raises(bits.BitsError) as ei:
        db.enumerate(a)
    assert ei.value.status == 6
    db.free()
    db = bits.Database(b, enumerate=True)
    off, _ = db.enumerate(a)
    assert off.cpu().tolist() == [0, 2, 3]
    # Offsets of other queries: the kernel notices the counts differ.
    pairs = torch.empty((3, 2), dtype=torch.uint32, device="cuda")
    other = dev(np.array([[0, 3], [6, 7]], np.uint32))
    lib = bits._lib.load()
    st = lib.bits_enumerate_pairs(db.handle, other.data_ptr(), 2, off.data_ptr(),
                                  pairs.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0
    with pytest.raises(bits.BitsError):
        db.check()
    # Inverted query: no pairs, error reported.
    with pytest.raises(bits.BitsError):
        db.enumerate(dev(np.array([[7, 6]], np.uint32)))
    db.free()
