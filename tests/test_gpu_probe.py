"""The random-read probe: the rate of random 64-byte node reads (diagnostic).

It is the hardware bound the search kernels are set against, so it must
separate an L2-resident buffer from a DRAM-sized one and give a rate of the
right order for each; bad arguments are codes, not faults.
"""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bits():
    from paper_1208_3407_b300 import probe
    return probe


def test_dram_rate_is_plausible_and_below_l2_rate(bits):
    dram = max(bits.probe_random_reads(4 << 30, 1 << 24) for _ in range(2))
    l2 = max(bits.probe_random_reads(32 << 20, 1 << 24) for _ in range(2))
    # Random 64-byte reads from HBM: between 1e9 and the 6.4 TB/s copy rate.
    assert 1e9 < dram < 6.4e12 / 64
    # A buffer inside the 126 MB L2 is served faster than one 30x larger.
    assert l2 > 1.5 * dram
    # Both halves of a random 128-byte line: at most the byte rate allows,
    # and no more accesses per second than single nodes.
    pairs = max(bits.probe_random_reads(4 << 30, 1 << 24, pairs=True) for _ in range(2))
    assert 1e9 < pairs < 6.4e12 / 128
    assert pairs < 1.1 * dram
    # The same lines read by one load instruction each: never slower than
    # two loads, and within the byte rate.
    line = max(bits.probe_random_reads(4 << 30, 1 << 24, pairs=True, one_load=True)
               for _ in range(2))
    assert 0.9 * pairs < line < 6.4e12 / 128


def test_argument_errors(bits):
    import ctypes as C
    lib = bits.load()
    buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    rate = C.c_double()
    assert lib.bits_probe_random_reads(buf.data_ptr(), 1000, 16, 1, C.byref(rate), None) == 1
    assert lib.bits_probe_random_reads(buf.data_ptr() + 16, 1 << 16, 16, 1, C.byref(rate),
                                       None) == 1
    assert lib.bits_probe_random_reads(buf.data_ptr() + 64, 1 << 16, 16, 2, C.byref(rate),
                                       None) == 1
    assert lib.bits_probe_random_reads(buf.data_ptr(), 1 << 20, 1 << 16, 1, C.byref(rate),
                                       None) == 0
    assert lib.bits_probe_random_reads(buf.data_ptr(), 1 << 20, 1 << 16, 2, C.byref(rate),
                                       None) == 0
    assert lib.bits_probe_random_reads(buf.data_ptr(), 1 << 20, 1 << 16, 3, C.byref(rate),
                                       None) == 0
    assert lib.bits_probe_random_reads(buf.data_ptr() + 64, 1 << 16, 16, 3, C.byref(rate),
                                       None) == 1
    assert rate.value > 0
