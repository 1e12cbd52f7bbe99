"""Parity of the database sort (B_S <- starts, B_E <- ends, each sorted:
Algorithm 2's two Sort steps) with the oracle's std::sort, bit for bit.

The cases reach every path of the keys-only one-sweep sort: tiles of 8192
keys with ragged last tiles (one key, one short of a tile, one past it),
full 32-bit keys (four passes), keys whose top digits are constant (passes
skipped; an odd number of passes ends with a copy out of the ping-pong
buffer), starts and ends with different numbers of active passes (one
array alone in the later passes), all keys equal (no pass at all), heavy
duplicates from clustered reads, warps whose 32 keys share one digit (the
peer tables' worst case), coordinates at 0 and 2^32 - 1, and the
allocation-free entry point writing to outputs that are only 4-byte
aligned (tiles then come through plain loads instead of bulk copies).
"""
import numpy as np
import pytest
import torch

import bits_synth as synth
import oracle

pytestmark = pytest.mark.gpu

O = oracle.get()


def intervals(rng, n, lo=0, hi=2**32 - 2, max_len=1000):
    s = rng.integers(lo, hi, size=n, dtype=np.int64)
    ln = rng.integers(1, max_len + 1, size=n, dtype=np.int64)
    e = np.minimum(s + ln, 2**32 - 1)
    return np.stack([s, e], axis=1).astype(np.uint32)


def check_build(b_np, **kw):
    import paper_1208_3407_b300 as bits
    db = bits.Database(torch.from_numpy(b_np).cuda(), **kw)
    gs, ge = db.sorted_arrays()
    gs, ge = gs.cpu().numpy().copy(), ge.cpu().numpy().copy()
    db.free()
    es, ee = O.build(b_np)
    np.testing.assert_array_equal(gs, es)
    np.testing.assert_array_equal(ge, ee)


@pytest.mark.parametrize("n", [1, 15, 8191, 8192, 8193, 3 * 16384 + 5, 1_000_003])
def test_full_range_keys_ragged_sizes(n):
    check_build(intervals(np.random.default_rng(n), n))


@pytest.mark.parametrize("hi,max_len", [(2**24 - 2000, 1000),    # top digit constant: 3 passes
                                        (2**16 - 300, 200),      # 2 passes
                                        (200, 50)])              # 1 pass
def test_skipped_passes(hi, max_len):
    check_build(intervals(np.random.default_rng(hi), 100_003, hi=hi, max_len=max_len))


def test_arrays_with_different_pass_counts():
    # starts below 2^16 (2 passes), ends spread over 32 bits (4 passes)
    rng = np.random.default_rng(5)
    n = 50_001
    s = rng.integers(0, 2**16, size=n, dtype=np.int64)
    e = s + rng.integers(1, 2**32 - 2**16 - 1, size=n, dtype=np.int64)
    check_build(np.stack([s, e], axis=1).astype(np.uint32))


def test_all_keys_equal_and_extremes():
    check_build(np.tile(np.array([[7, 9]], np.uint32), (20_000, 1)))
    b = np.array([[0, 1], [0, 2**32 - 1], [2**32 - 2, 2**32 - 1], [5, 6]] * 5000, np.uint32)
    check_build(b)


def test_warps_sharing_one_digit():
    # The first pass sees the keys in input order: each run of 32 (one warp's
    # slot of a tile) has one low digit, every fifth run two digits by lane
    # parity, so the peer tables see all 32 lanes (or 16) on one word.  The
    # upper bytes are random, so all four passes run.
    rng = np.random.default_rng(17)
    n = 3 * 8192 + 4099
    i = np.arange(n, dtype=np.int64)
    low = (i // 32) % 256
    alt = ((i // 32) % 5 == 0) & (i % 2 == 1)
    low = np.where(alt, (low + 128) % 256, low)
    s = (rng.integers(0, 2**23, size=n, dtype=np.int64) << 8) | low
    e = s + rng.integers(1, 256, size=n, dtype=np.int64)
    b = np.stack([s, e], axis=1).astype(np.uint32)
    check_build(b)
    check_build(b, enumerate=True)   # the key/value sort ranks the same way


def test_clustered_duplicates_at_scale():
    _, _, b = synth.config2(n_a=1, n_b=3_000_000, n_hot=2000, seed_b=41)
    check_build(b)
    check_build(b, enumerate=True)   # the key/value sort of the enumeration table


def test_noalloc_with_4_byte_aligned_outputs():
    from paper_1208_3407_b300 import _lib
    lib = _lib.load()
    b_np = intervals(np.random.default_rng(9), 100_000)
    n = b_np.shape[0]
    b = torch.from_numpy(b_np).cuda()
    buf_s = torch.zeros(n + 4, dtype=torch.uint32, device="cuda")
    buf_e = torch.zeros(n + 4, dtype=torch.uint32, device="cuda")
    st = lib.bits_sort_intervals_noalloc(b.data_ptr(), n, buf_s.data_ptr() + 4,
                                         buf_e.data_ptr() + 12, None)
    assert st == _lib.BITS_OK, lib.bits_last_error()
    torch.cuda.synchronize()
    es, ee = O.build(b_np)
    np.testing.assert_array_equal(buf_s[1:n + 1].cpu().numpy(), es)
    np.testing.assert_array_equal(buf_e[3:n + 3].cpu().numpy(), ee)
