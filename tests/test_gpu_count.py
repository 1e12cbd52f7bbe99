"""Parity of the CUDA sort and count path with the CPU oracle (bit-exact).

Every case builds the database on the GPU through the C ABI and compares
the sorted arrays, every per-query count and the total with the oracle on
the same seeded inputs.
"""
import numpy as np
import pytest
import torch

import bits_synth as synth
import oracle
from goldens import read_count_fixture

pytestmark = pytest.mark.gpu

O = oracle.get()


def dev(x: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def bits():
    import paper_1208_3407_b300 as bits
    return bits


def gpu_count(bits, a, b, **kw):
    method = kw.pop("method", None)
    db = bits.Database(dev(b), **kw)
    counts, total = db.count(dev(a), method=method)
    torch.cuda.synchronize()
    out = host(counts), int(host(total)[0])
    bs, be = db.sorted_arrays()
    arrays = host(bs).copy(), host(be).copy()
    db.free()
    return out, arrays


def assert_parity(bits, a, b, check_sort=True, **kw):
    (c, t), (bs, be) = gpu_count(bits, a, b, **kw)
    obs, obe = O.build(b)
    if check_sort:
        np.testing.assert_array_equal(bs, obs)
        np.testing.assert_array_equal(be, obe)
    oc, ot = O.count_sorted(a, obs, obe)
    np.testing.assert_array_equal(c, oc)
    assert t == ot


@pytest.mark.parametrize("name", ["containment.txt", "duplicates.txt"])
def test_golden_fixture(bits, name):
    a, b, exp, total = read_count_fixture(name)
    (c, t), _ = gpu_count(bits, a, b)
    np.testing.assert_array_equal(c, exp)
    assert t == total


def test_config1_full_against_brute_force(bits):
    a, b = synth.config1()
    (c, t), _ = gpu_count(bits, a, b)
    bc, bt = O.count_brute(a, b)
    np.testing.assert_array_equal(c, bc)
    assert t == bt


@pytest.mark.parametrize("seed", range(40))
def test_tiny_random(bits, seed):
    rng = np.random.default_rng(seed)
    na, nb = int(rng.integers(1, 300)), int(rng.integers(1, 300))
    a, b = synth.tiny_random(seed, na, nb, coord_max=int(rng.integers(4, 400)),
                             max_len=int(rng.integers(1, 40)))
    t = int(rng.integers(2, 9))
    (c, tot), _ = gpu_count(bits, a, b, top_tree_log2=t)
    bc, bt = O.count_brute(a, b)
    np.testing.assert_array_equal(c, bc)
    assert tot == bt


@pytest.mark.parametrize("nb", [1, 2, 7, 8191, 8192, 8193, 3 * 8192 + 5, 100_003])
def test_sort_sizes_and_ragged_tiles(bits, nb):
    _, a, b = synth.config2(n_a=1001, n_b=nb, n_hot=max(1, nb // 10))
    assert_parity(bits, a, b)


def test_config2_reduced_all_tree_depths(bits):
    _, a, b = synth.config2(n_a=20_001, n_b=2_000_000, n_hot=20_000)
    for t in (2, 6, 13, 14):
        assert_parity(bits, a, b, check_sort=(t == 13), top_tree_log2=t)


def test_config2_full(bits):
    _, a, b = synth.config2()
    assert_parity(bits, a, b)


@pytest.mark.parametrize("top", [2, 12])
def test_long_and_short_queries_share_octets(bits, top):
    # The count kernel reads a query's starts node and ends node of a level
    # with one load by eight lanes.  Point-like queries keep the two ranks in
    # one node; queries spanning a quarter of the line separate them on every
    # level.  Mixed lane by lane, with a ragged last octet and warp.
    rng = np.random.default_rng(91)
    nb = 200_000
    bs = rng.integers(0, 1 << 31, nb, dtype=np.uint64)
    b = np.stack([bs, bs + 1 + rng.integers(0, 100_000, nb, dtype=np.uint64)], 1)
    na = 8 * 1237 + 5
    s = rng.integers(0, 1 << 31, na, dtype=np.uint64)
    lens = np.where(np.arange(na) % 3 == 0, rng.integers(1 << 24, 1 << 30, na, dtype=np.uint64),
                    rng.integers(1, 10, na, dtype=np.uint64))
    a = np.stack([s, s + lens], 1)
    assert_parity(bits, a.astype(np.uint32), b.astype(np.uint32), check_sort=False,
                  top_tree_log2=top)


def test_constant_digits_are_skipped_correctly(bits):
    # Keys < 2^24 (top digit constant), and a database of identical intervals
    # (every digit constant).
    a, b = synth.config1(n_a=5000, n_b=70_000)
    assert_parity(bits, a, b)
    same = np.tile(np.array([[123456, 123999]], np.uint32), (20_000, 1))
    assert_parity(bits, a, same)


def test_empty_inputs(bits):
    a, b = synth.config1(n_a=100, n_b=100)
    (c, t), _ = gpu_count(bits, a, np.zeros((0, 2), np.uint32))
    assert t == 0 and (c == 0).all()
    (c, t), _ = gpu_count(bits, np.zeros((0, 2), np.uint32), b)
    assert t == 0 and c.shape == (0,)


def test_odd_and_misaligned_query_pointers(bits):
    _, a, b = synth.config2(n_a=4097, n_b=50_000, n_hot=100)
    db = bits.Database(dev(b))
    obs, obe = O.build(b)
    da = dev(a)
    for lo in (0, 1, 3):
        sub = da[lo:]
        c, t = db.count(sub)
        oc, ot = O.count_sorted(a[lo:], obs, obe)
        np.testing.assert_array_equal(host(c), oc)
        assert int(host(t)[0]) == ot
    # counts into a misaligned output slice
    buf = torch.zeros(a.shape[0] + 1, dtype=torch.uint32, device="cuda")
    c, t = db.count(da, counts=buf[1:])
    np.testing.assert_array_equal(host(buf[1:]), O.count_sorted(a, obs, obe)[0])
    db.free()


def test_total_only(bits):
    _, a, b = synth.config2(n_a=10_000, n_b=100_000, n_hot=100)
    db = bits.Database(dev(b))
    c, t = db.count(dev(a), counts=False)
    assert c is None
    assert int(host(t)[0]) == O.count(a, b)[1]
    db.free()


def test_extreme_coordinates(bits):
    top = 2**32 - 1
    b = np.array([[top - 5, top], [0, 1], [top - 1, top]], np.uint32)
    a = np.array([[top - 1, top - 1], [top - 2, top], [top, top], [0, 0], [0, top]], np.uint32)
    (c, t), _ = gpu_count(bits, a, b)
    np.testing.assert_array_equal(c, O.count_brute(a, b)[0])
    b2 = np.concatenate([b, synth.config1(n_b=30_000)[1]])
    a2 = np.concatenate([a, synth.config1(n_a=3000)[0]])
    assert_parity(bits, a2, b2)


def test_invariants_on_gpu(bits):
    _, a, b = synth.config3(n_a=30_000, n_b=60_000, n_hot=500)
    (_, t_ab), _ = gpu_count(bits, a, b)
    (_, t_ba), _ = gpu_count(bits, b, a)
    assert t_ab == t_ba
    shift = np.uint32(1000)
    (_, t_sh), _ = gpu_count(bits, a + shift, b + shift)
    assert t_sh == t_ab


def test_inverted_query_is_reported(bits):
    b = synth.config1(n_b=1000)[1]
    db = bits.Database(dev(b))
    a = np.array([[10, 20], [30, 25], [40, 50]], np.uint32)
    with pytest.raises(bits.BitsError) as e:
        db.count(dev(a))
    assert e.value.status == 1
    # The error word is cleared: a valid call succeeds afterwards.
    c, t = db.count(dev(a[[0, 2]]))
    db.free()


def test_invalid_database_is_rejected(bits):
    b = np.array([[5, 10], [7, 7], [1, 2]], np.uint32)
    with pytest.raises(bits.BitsError) as e:
        bits.Database(dev(b))
    assert e.value.status == 1


def test_side_stream(bits):
    _, a, b = synth.config2(n_a=5000, n_b=300_000, n_hot=1000)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        db = bits.Database(dev(b), stream=s)
        c, t = db.count(dev(a), stream=s)
    s.synchronize()
    oc, ot = O.count(a, b)
    np.testing.assert_array_equal(host(c), oc)
    db.free()
