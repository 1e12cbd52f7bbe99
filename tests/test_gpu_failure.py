"""Failure detection without a GPU fault: bounded waits and bad inputs.

A wait that nothing ends must give up with BITS_ETIMEOUT and leave the
context usable; invalid inputs must come back as error codes, not faults.
"""
import numpy as np
import pytest
import torch

import bits_synth as synth
import oracle

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import paper_1208_3407_b300 as bits
    from paper_1208_3407_b300 import _lib
    lib = _lib.load()
    st = torch.cuda.current_stream().cuda_stream
    assert lib.bits_selftest_wait(20_000, st) == _lib.BITS_ETIMEOUT
    assert b"ran out" in lib.bits_last_error()
    assert lib.bits_selftest_wait(0, st) == _lib.BITS_EINVAL
    # the context is still usable: a count right after is exact
    a, b = synth.config1(n_a=2000, n_b=3000)
    db = bits.Database(torch.from_numpy(b).cuda())
    c, t = db.count(torch.from_numpy(a).cuda())
    np.testing.assert_array_equal(c.cpu().numpy(), oracle.get().count_brute(a, b)[0])
    db.free()


def test_bad_arguments_are_codes_not_faults():
    import paper_1208_3407_b300 as bits
    from paper_1208_3407_b300 import _lib
    lib = _lib.load()
    b = torch.from_numpy(synth.config1(n_b=100)[1]).cuda()
    db = bits.Database(b)
    a = torch.zeros((4, 2), dtype=torch.uint32, device="cuda")
    tot = torch.zeros(1, dtype=torch.uint64, device="cuda")
    # misaligned query pointer (4 bytes into the tensor)
    assert lib.bits_count(db.handle, a.data_ptr() + 4, 2, None, tot.data_ptr(), None) == _lib.BITS_EINVAL
    assert lib.bits_count_method(db.handle, 9, a.data_ptr(), 2, None, tot.data_ptr(), None) == _lib.BITS_EINVAL
    assert lib.bits_count_method(db.handle, bits.METHOD_RMI, a.data_ptr(), 2, None, tot.data_ptr(),
                                 None) == _lib.BITS_ENOTIMPL
    assert lib.bits_count(db.handle, a.data_ptr(), 1 << 32, None, tot.data_ptr(), None) == _lib.BITS_EOVERFLOW
    db.free()
