"""bits_count_host: the count end to end on host buffers, bit-exact with the oracle.

Page-locked inputs and outputs are read and written in place by the search
kernel; pageable ones are staged by the library.  Every case compares every
per-query count and the total with the CPU oracle on the same seeded inputs.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import bits_synth as synth
import oracle

pytestmark = pytest.mark.gpu

O = oracle.get()


def dev(x: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32)).cuda()


def pinned(x: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32)).pin_memory()


@pytest.fixture(scope="module")
def bits():
    import paper_1208_3407_b300 as bits
    return bits


@pytest.fixture(scope="module")
def case(bits):
    _, a, b = synth.config2(n_a=70_001, n_b=1_000_003, n_hot=10_000)
    db = bits.Database(dev(b), rmi_leaves_log2=12)
    obs, obe = O.build(b)
    oc, ot = O.count_sorted(a, obs, obe)
    yield db, a, b, oc, ot
    db.free()


@pytest.mark.parametrize("method", [0, 1, 2, 3])
@pytest.mark.parametrize("n", [0, 1, 31, 4097, 70_001])
def test_pinned_in_place(bits, case, method, n):
    db, a, _, oc, _ = case
    c, t = db.count_host(pinned(a[:n]), method=method)
    assert c.is_pinned() or n == 0
    np.testing.assert_array_equal(c.numpy(), oc[:n])
    assert t == int(oc[:n].sum(dtype=np.uint64))


@pytest.mark.parametrize("method", [1, 2, 3])
def test_pageable_is_staged(bits, case, method):
    db, a, _, oc, ot = case
    out = np.full(a.shape[0], 7, np.uint32)
    c, t = db.count_host(np.ascontiguousarray(a), counts=out, method=method)
    np.testing.assert_array_equal(out, oc)
    assert t == ot


def test_mixed_pinned_and_pageable(bits, case):
    db, a, _, oc, ot = case
    out = np.zeros(a.shape[0], np.uint32)
    _, t = db.count_host(pinned(a), counts=out, method=1)
    np.testing.assert_array_equal(out, oc)
    assert t == ot
    out_p = torch.zeros(a.shape[0], dtype=torch.uint32).pin_memory()
    _, t = db.count_host(np.ascontiguousarray(a), counts=out_p, method=1)
    np.testing.assert_array_equal(out_p.numpy(), oc)
    assert t == ot


def test_offset_views_and_total_only(bits, case):
    db, a, _, oc, ot = case
    big = torch.zeros((a.shape[0] + 3, 2), dtype=torch.uint32).pin_memory()
    big[3:] = torch.from_numpy(a)
    cbuf = torch.zeros(a.shape[0] + 1, dtype=torch.uint32).pin_memory()
    _, t = db.count_host(big[3:], counts=cbuf[1:], method=1)
    np.testing.assert_array_equal(cbuf[1:].numpy(), oc)
    assert cbuf[0].item() == 0 and t == ot
    c, t = db.count_host(pinned(a), counts=None, method=1)
    assert c is None and t == ot


def test_async_calls_on_two_streams(bits, case):
    # Page-locked buffers everywhere: both calls return at once, each adds
    # into a device word of its own, and the results are in place after a
    # synchronisation.
    db, a, _, oc, _ = case
    h = pinned(a)
    n = a.shape[0]
    outs = [torch.zeros(n, dtype=torch.uint32).pin_memory() for _ in range(2)]
    tots = [torch.zeros(1, dtype=torch.uint64).pin_memory() for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for k, s in enumerate(streams):
        db.count_host(h[1000 * k:], counts=outs[k], total=tots[k], method=1, stream=s,
                      check=False)
    torch.cuda.synchronize()
    for k in range(2):
        np.testing.assert_array_equal(outs[k].numpy()[:n - 1000 * k], oc[1000 * k:])
        assert int(tots[k].numpy()[0]) == int(oc[1000 * k:].sum(dtype=np.uint64))
    db.check()


def test_matches_device_path_on_exome_vs_reads(bits):
    _, a, b = synth.config2()
    db = bits.Database(dev(b))
    dc, dt = db.count(dev(a), method=1)
    c, t = db.count_host(pinned(a), method=1)
    np.testing.assert_array_equal(c.numpy(), dc.cpu().numpy())
    assert t == int(dt.cpu().numpy()[0])
    idx = np.random.default_rng(5).choice(a.shape[0], size=512, replace=False)
    oc, _ = O.count_brute(a[idx], b)
    np.testing.assert_array_equal(c.numpy()[idx], oc)
    db.free()


def test_inverted_query_and_errors(bits, case):
    db, a, _, oc, _ = case
    bad = a[:100].copy()
    bad[17] = [50, 40]
    with pytest.raises(bits.BitsError) as e:
        db.count_host(pinned(bad), method=1)
    assert e.value.status == 1
    c, t = db.count_host(pinned(a[:100]), method=1)      # error word was cleared
    np.testing.assert_array_equal(c.numpy(), oc[:100])
    with pytest.raises(TypeError):
        db.count_host(dev(a[:10]))
    lib = db._lib
    tot = C.c_uint64()
    d = dev(a[:10])
    assert lib.bits_count_host(db.handle, 1, d.data_ptr(), 10, None, C.byref(tot), None) == 1
    h = pinned(a[:10])
    assert lib.bits_count_host(db.handle, 9, h.data_ptr(), 10, None, C.byref(tot), None) == 1
    assert lib.bits_count_host(db.handle, 1, h.data_ptr() + 4, 9, None, C.byref(tot), None) == 1
    assert lib.bits_count_host(db.handle, 1, h.data_ptr(), 10, None, None, None) == 1


def test_database_without_learned_index(bits):
    _, a, b = synth.config2(n_a=1000, n_b=20_000, n_hot=100)
    db = bits.Database(dev(b))
    with pytest.raises(bits.BitsError) as e:
        db.count_host(pinned(a), method=2)
    assert e.value.status == 6
    c, t = db.count_host(pinned(a))                       # AUTO
    np.testing.assert_array_equal(c.numpy(), O.count(a, b)[0])
    db.free()
