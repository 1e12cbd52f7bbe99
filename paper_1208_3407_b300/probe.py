"""Binding of libbits_probe.so (include/bits_probe.h): the random-read probe.

A measurement aid, not part of the method: the benchmark measures with it
the rate at which this GPU serves random 64-byte node reads (from DRAM on a
buffer much larger than L2, from L2 on a small one), the hardware bound the
search kernels are set against.  Loading fails loudly when the library is
missing.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import _lib

LIB_PATH = os.path.join(_lib.HERE, "libbits_probe.so")
EXPORTS = ["bits_probe_random_reads"]

_probe = None


def load():
    global _probe
    if _probe is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1208_3407_b300.build` (nvcc, sm_103a)")
        _lib.load()  # the probe library resolves its error reporting from the main library
        lib = C.CDLL(LIB_PATH)
        lib.bits_probe_random_reads.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int32,
                                                C.POINTER(C.c_double), C.c_void_p]
        lib.bits_probe_random_reads.restype = C.c_int
        _probe = lib
    return _probe


def probe_random_reads(nbytes: int = 4 << 30, n_reads: int = 1 << 24, *, pairs: bool = False,
                       one_load: bool = False, device=None, stream=None) -> float:
    """bits_probe_random_reads on a fresh ``nbytes`` device buffer: random
    accesses per second, each one 64-byte node (access kind 1), or, with
    ``pairs``, both halves of one 128-byte line read by two loads (kind 2) or,
    with ``one_load`` as well, by one load instruction (kind 3)."""
    if one_load and not pairs:
        raise ValueError("one_load reads a whole 128-byte line: it needs pairs=True")
    kind = (3 if one_load else 2) if pairs else 1
    buf = torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")
    rate = C.c_double()
    s = stream if stream is not None else torch.cuda.current_stream(buf.device)
    with torch.cuda.device(buf.device):
        _lib.check(load().bits_probe_random_reads(buf.data_ptr(), nbytes, n_reads, kind,
                                                  C.byref(rate), int(s.cuda_stream)),
                   "bits_probe_random_reads")
    del buf
    return rate.value
