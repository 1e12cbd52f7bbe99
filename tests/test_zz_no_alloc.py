"""The allocation-free sort entry point, checked against the CPU oracle.

bits_sort_intervals_noalloc exists for callers that cannot allocate device
memory -- code whose GPU memory is owned by another allocator, or serving
loops that fix their memory plan up front.  It keeps its scratch in a fixed
array inside the library instead of calling cudaMalloc.  These tests call it
through the C ABI:
  * twice in a row (a larger then a smaller input, so stale scratch contents
    from the first call would show up in the second), comparing both outputs
    bit-exactly with the oracle's std::sort of the same starts and ends, and
    with the arrays bits_build_db sorts;
  * with the device's free memory read before and after a call (it must not
    change: the call allocates nothing);
  * with an inverted interval, which must give BITS_EINVAL, followed by a
    valid call that must succeed with correct output (the error word is
    cleared per call);
  * with a size beyond the fixed scratch, which must be refused.
The file is named to be collected last.
"""
import numpy as np
import pytest
import torch

import bits_synth as synth
import oracle

pytestmark = pytest.mark.gpu

MAX_N = 262144
O = oracle.get()


def _sort(lib, b: torch.Tensor, out_s: torch.Tensor, out_e: torch.Tensor) -> int:
    stream = torch.cuda.current_stream()
    return lib.bits_sort_intervals_noalloc(b.data_ptr(), b.shape[0], out_s.data_ptr(),
                                           out_e.data_ptr(), stream.cuda_stream)


def test_noalloc_sort_matches_oracle_on_two_calls_in_a_row():
    import paper_1208_3407_b300 as bits
    from paper_1208_3407_b300 import _lib

    lib = _lib.load()
    cases = [synth.config2(n_a=1, n_b=250_001, n_hot=3000, seed_b=31)[2],
             synth.config3(n_a=1, n_b=77_777, n_hot=500, seed_b=32)[2]]
    for b_np in cases:
        n = b_np.shape[0]
        b = torch.from_numpy(b_np).cuda()
        out_s = torch.full((n,), 7, dtype=torch.uint32, device="cuda")
        out_e = torch.full((n,), 7, dtype=torch.uint32, device="cuda")
        st = _sort(lib, b, out_s, out_e)
        assert st == _lib.BITS_OK, lib.bits_last_error()
        torch.cuda.synchronize()
        exp_s, exp_e = O.build(b_np)
        np.testing.assert_array_equal(out_s.cpu().numpy(), exp_s)
        np.testing.assert_array_equal(out_e.cpu().numpy(), exp_e)
        db = bits.Database(b)
        ref_s, ref_e = db.sorted_arrays()
        np.testing.assert_array_equal(out_s.cpu().numpy(), ref_s.cpu().numpy())
        np.testing.assert_array_equal(out_e.cpu().numpy(), ref_e.cpu().numpy())
        db.free()


def test_noalloc_sort_allocates_nothing():
    from paper_1208_3407_b300 import _lib

    lib = _lib.load()
    b_np = synth.config3(n_a=1, n_b=MAX_N, n_hot=2000, seed_b=33)[2]
    b = torch.from_numpy(b_np).cuda()
    out_s = torch.empty(MAX_N, dtype=torch.uint32, device="cuda")
    out_e = torch.empty(MAX_N, dtype=torch.uint32, device="cuda")
    assert _sort(lib, b, out_s, out_e) == _lib.BITS_OK, lib.bits_last_error()  # warm-up
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    out_s.fill_(0)
    out_e.fill_(0)
    torch.cuda.synchronize()
    assert _sort(lib, b, out_s, out_e) == _lib.BITS_OK, lib.bits_last_error()
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    exp_s, exp_e = O.build(b_np)
    np.testing.assert_array_equal(out_s.cpu().numpy(), exp_s)
    np.testing.assert_array_equal(out_e.cpu().numpy(), exp_e)


def test_noalloc_sort_rejects_inverted_then_recovers():
    from paper_1208_3407_b300 import _lib

    lib = _lib.load()
    b_np = synth.config1(n_a=1, n_b=5000)[1]
    bad = b_np.copy()
    bad[1234] = [500, 500]                     # end <= start: not a database interval
    n = bad.shape[0]
    out_s = torch.empty(n, dtype=torch.uint32, device="cuda")
    out_e = torch.empty(n, dtype=torch.uint32, device="cuda")
    st = _sort(lib, torch.from_numpy(bad).cuda(), out_s, out_e)
    assert st == _lib.BITS_EINVAL
    assert b"end <= start" in lib.bits_last_error()
    st = _sort(lib, torch.from_numpy(b_np).cuda(), out_s, out_e)
    assert st == _lib.BITS_OK, lib.bits_last_error()
    torch.cuda.synchronize()
    exp_s, exp_e = O.build(b_np)
    np.testing.assert_array_equal(out_s.cpu().numpy(), exp_s)
    np.testing.assert_array_equal(out_e.cpu().numpy(), exp_e)


def test_noalloc_sort_rejects_sizes_beyond_its_scratch():
    from paper_1208_3407_b300 import _lib

    lib = _lib.load()
    dummy = torch.zeros(8, dtype=torch.uint32, device="cuda")
    st = lib.bits_sort_intervals_noalloc(dummy.data_ptr(), MAX_N + 1, dummy.data_ptr(),
                                         dummy.data_ptr(), None)
    assert st == _lib.BITS_EOVERFLOW
    assert b"BITS_NOALLOC_MAX_INTERVALS" in lib.bits_last_error()
