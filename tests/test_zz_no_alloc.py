"""The allocation-free sort entry point gives the same arrays as bits_build_db.

bits_sort_intervals_noalloc exists for callers that cannot allocate device
memory -- code whose GPU memory is owned by another allocator, or serving
loops that fix their memory plan up front.  It keeps its scratch in a fixed
array inside the library instead of calling cudaMalloc.  This test calls it
through the C ABI twice in a row (a larger then a smaller input, so stale
scratch contents from the first call would show up in the second) and
compares both outputs bit-exactly with the sorted arrays bits_build_db
produces for the same intervals.  The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import bits_synth as synth

pytestmark = pytest.mark.gpu

MAX_N = 262144


def test_noalloc_sort_matches_build_db_on_two_calls_in_a_row():
    import paper_1208_3407_b300 as bits
    from paper_1208_3407_b300 import _lib

    lib = _lib.load()
    stream = torch.cuda.current_stream()
    cases = [synth.config2(n_a=1, n_b=250_001, n_hot=3000, seed_b=31)[2],
             synth.config3(n_a=1, n_b=77_777, n_hot=500, seed_b=32)[2]]
    for b_np in cases:
        n = b_np.shape[0]
        b = torch.from_numpy(b_np).cuda()
        out_s = torch.full((n,), 7, dtype=torch.uint32, device="cuda")
        out_e = torch.full((n,), 7, dtype=torch.uint32, device="cuda")
        st = lib.bits_sort_intervals_noalloc(b.data_ptr(), n, out_s.data_ptr(), out_e.data_ptr(),
                                             stream.cuda_stream)
        assert st == _lib.BITS_OK, lib.bits_last_error()
        db = bits.Database(b)
        ref_s, ref_e = db.sorted_arrays()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out_s.cpu().numpy(), ref_s.cpu().numpy())
        np.testing.assert_array_equal(out_e.cpu().numpy(), ref_e.cpu().numpy())
        db.free()


def test_noalloc_sort_rejects_sizes_beyond_its_scratch():
    from paper_1208_3407_b300 import _lib

    lib = _lib.load()
    dummy = torch.zeros(8, dtype=torch.uint32, device="cuda")
    st = lib.bits_sort_intervals_noalloc(dummy.data_ptr(), MAX_N + 1, dummy.data_ptr(),
                                         dummy.data_ptr(), None)
    assert st == _lib.BITS_EOVERFLOW
    assert b"BITS_NOALLOC_MAX_INTERVALS" in lib.bits_last_error()
