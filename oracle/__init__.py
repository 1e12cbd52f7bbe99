"""ctypes wrapper around the CPU oracle (``bits_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
benchmark's CPU-baseline leg use it.  The CUDA library never imports it and
it never imports the CUDA library.

Interval sets are ``(n, 2)`` ``numpy.uint32`` arrays of half-open
``[start, end)`` pairs.  Every function raises ``ValueError`` when the oracle
rejects its input (inverted query, empty or inverted database interval,
interval outside its contig).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bits_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(out: str = _LIB, defines: tuple[str, ...] = ()) -> str:
    """Compile the oracle with g++ (no CUDA involved)."""
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, "-o", out]
    cmd += [f"-D{d}" for d in defines]
    subprocess.run(cmd, check=True)
    return out


def _stale() -> bool:
    return (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)


def _declare(lib):
    u32p, u64p = C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)
    lib.or_count_brute.argtypes = [u32p, C.c_uint64, u32p, C.c_uint64, u32p, u64p]
    lib.or_build.argtypes = [u32p, C.c_uint64, u32p, u32p]
    lib.or_count_sorted.argtypes = [u32p, C.c_uint64, u32p, u32p, C.c_uint64, u32p, u64p, C.c_int]
    lib.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.or_philox4x32_10.restype = None
    lib.or_scale_u64.argtypes = [C.c_uint64, C.c_uint64]
    lib.or_scale_u64.restype = C.c_uint64
    lib.or_mc_place.argtypes = [u32p, C.c_uint64, u32p, u32p, C.c_uint32, C.c_uint64, C.c_uint32, u32p]
    lib.or_mc.argtypes = [u32p, C.c_uint64, u32p, u32p, C.c_uint32, u32p, u32p, C.c_uint64,
                          C.c_uint64, C.c_uint32, C.c_uint32, u64p, u64p, u64p,
                          C.POINTER(C.c_double), C.c_int]
    lib.or_mc_place_set.argtypes = [u32p, C.c_uint64, u32p, u32p, C.c_uint32, C.c_uint64, C.c_uint32,
                                    C.c_uint32, u32p]
    lib.or_mc_set.argtypes = [u32p, C.c_uint64, u32p, u32p, C.c_uint32, u32p, u32p, C.c_uint64,
                              C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, u64p, u64p, u64p,
                              C.POINTER(C.c_double), C.c_int]
    lib.or_mc_summary.argtypes = [u64p, C.c_uint64, C.c_uint64, u64p, C.POINTER(C.c_double)]
    lib.or_enumerate_brute.argtypes = [u32p, C.c_uint64, u32p, C.c_uint64, u64p, u32p]
    lib.or_enumerate_scan.argtypes = [u32p, C.c_uint64, u32p, C.c_uint64, u64p, u32p]
    lib.or_count_brute_closed.argtypes = [u32p, C.c_uint64, u32p, C.c_uint64, u32p, u64p]
    lib.or_project.argtypes = [u32p, u32p, u32p, C.c_uint64, u32p, u32p, C.c_uint32, C.c_int, u32p]
    lib.or_project.restype = C.c_uint64
    for f in ("or_count_brute", "or_build", "or_count_sorted", "or_mc_place", "or_mc",
              "or_count_brute_closed", "or_mc_place_set", "or_mc_set", "or_mc_summary",
              "or_enumerate_brute", "or_enumerate_scan"):
        getattr(lib, f).restype = C.c_int
    return lib


def load(path: str | None = None):
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if path is not None:
        return _declare(C.CDLL(path))
    with _lock:
        if _lib is None:
            if _stale():
                build()
            _lib = _declare(C.CDLL(_LIB))
    return _lib


def _p32(x: np.ndarray):
    assert x.dtype == np.uint32 and x.flags.c_contiguous
    return x.ctypes.data_as(C.POINTER(C.c_uint32))


def _p64(x: np.ndarray):
    assert x.dtype == np.uint64 and x.flags.c_contiguous
    return x.ctypes.data_as(C.POINTER(C.c_uint64))


def _iv(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint32)
    return x.reshape(-1, 2)


class Oracle:
    """Object form so a test can point it at a differently compiled library."""

    def __init__(self, lib=None):
        self.lib = lib or load()

    def count_brute(self, a, b):
        a, b = _iv(a), _iv(b)
        counts = np.zeros(a.shape[0], np.uint32)
        total = np.zeros(1, np.uint64)
        if self.lib.or_count_brute(_p32(a), a.shape[0], _p32(b), b.shape[0], _p32(counts), _p64(total)):
            raise ValueError("oracle rejected input")
        return counts, int(total[0])

    def count_brute_closed(self, a, b):
        """The closed predicate of Sec. "Interval Set Intersection problem", by
        brute force (intervals [start, end])."""
        a, b = _iv(a), _iv(b)
        counts = np.zeros(a.shape[0], np.uint32)
        total = np.zeros(1, np.uint64)
        if self.lib.or_count_brute_closed(_p32(a), a.shape[0], _p32(b), b.shape[0], _p32(counts),
                                          _p64(total)):
            raise ValueError("oracle rejected input")
        return counts, int(total[0])

    def project(self, chrom, start, end, contig_off=None, contig_len=None, closed=False):
        """The projection of Sec. "BITS Algorithm"; returns (intervals, number
        rejected).  Rejected rows are (2^32 - 1, 0).  With no contig table the line is one contig at 0."""
        start = np.ascontiguousarray(start, np.uint32)
        end = np.ascontiguousarray(end, np.uint32)
        n = start.shape[0]
        chrom = np.ascontiguousarray(np.zeros(n) if chrom is None else chrom, np.uint32)
        co = np.ascontiguousarray([] if contig_off is None else contig_off, np.uint32)
        cl = np.ascontiguousarray([] if contig_len is None else contig_len, np.uint32)
        out = np.zeros((n, 2), np.uint32)
        nil = C.cast(0, C.POINTER(C.c_uint32))
        bad = self.lib.or_project(_p32(chrom), _p32(start), _p32(end), n,
                                  _p32(co) if co.size else nil, _p32(cl) if cl.size else nil,
                                  co.shape[0], 1 if closed else 0, _p32(out))
        return out, int(bad)

    def _enumerate(self, fn, a, b):
        a, b = _iv(a), _iv(b)
        off = np.zeros(a.shape[0] + 1, np.uint64)
        nil = C.cast(0, C.POINTER(C.c_uint32))
        if fn(_p32(a), a.shape[0], _p32(b), b.shape[0], _p64(off), nil):
            raise ValueError("oracle rejected input")
        pairs = np.zeros((int(off[-1]), 2), np.uint32)
        fn(_p32(a), a.shape[0], _p32(b), b.shape[0], _p64(off), _p32(pairs) if pairs.size else nil)
        return off, pairs

    def enumerate_brute(self, a, b):
        """(offsets uint64[n+1], pairs uint32[total, 2]) by the definition, (i, j) order."""
        return self._enumerate(self.lib.or_enumerate_brute, a, b)

    def enumerate_scan(self, a, b):
        """Same pairs by the start-sorted scan terminated at ICount, in scan order."""
        return self._enumerate(self.lib.or_enumerate_scan, a, b)

    def build(self, b):
        b = _iv(b)
        bs = np.empty(b.shape[0], np.uint32)
        be = np.empty(b.shape[0], np.uint32)
        if self.lib.or_build(_p32(b), b.shape[0], _p32(bs), _p32(be)):
            raise ValueError("oracle rejected database")
        return bs, be

    def count_sorted(self, a, bs, be, threads: int = 1, want_counts: bool = True):
        a = _iv(a)
        bs = np.ascontiguousarray(bs, np.uint32)
        be = np.ascontiguousarray(be, np.uint32)
        counts = np.zeros(a.shape[0], np.uint32) if want_counts else None
        total = np.zeros(1, np.uint64)
        cp = _p32(counts) if want_counts else None
        if self.lib.or_count_sorted(_p32(a), a.shape[0], _p32(bs), _p32(be), bs.shape[0], cp,
                                    _p64(total), threads):
            raise ValueError("oracle rejected queries")
        return counts, int(total[0])

    def count(self, a, b, threads: int = 1):
        bs, be = self.build(b)
        return self.count_sorted(a, bs, be, threads)

    def philox(self, ctr, key):
        ctr = np.ascontiguousarray(ctr, np.uint32)
        key = np.ascontiguousarray(key, np.uint32)
        out = np.zeros(4, np.uint32)
        self.lib.or_philox4x32_10(_p32(ctr), _p32(key), _p32(out))
        return out

    def scale_u64(self, u: int, n: int) -> int:
        return int(self.lib.or_scale_u64(u, n))

    def mc_place(self, a, contig_off, contig_len, seed: int, s: int, set_index: int = 0):
        a = _iv(a)
        co = np.ascontiguousarray(contig_off, np.uint32)
        cl = np.ascontiguousarray(contig_len, np.uint32)
        out = np.zeros_like(a)
        if self.lib.or_mc_place_set(_p32(a), a.shape[0], _p32(co), _p32(cl), co.shape[0], seed, s,
                                    set_index, _p32(out)):
            raise ValueError("oracle rejected MC input")
        return out

    def mc(self, a, contig_off, contig_len, bs, be, seed: int, s_begin: int, s_end: int,
           threads: int = 1, set_index: int = 0):
        a = _iv(a)
        co = np.ascontiguousarray(contig_off, np.uint32)
        cl = np.ascontiguousarray(contig_len, np.uint32)
        bs = np.ascontiguousarray(bs, np.uint32)
        be = np.ascontiguousarray(be, np.uint32)
        totals = np.zeros(max(0, s_end - s_begin), np.uint64)
        obs = np.zeros(1, np.uint64)
        k = np.zeros(1, np.uint64)
        p = C.c_double(0.0)
        tp = _p64(totals) if totals.size else C.cast(0, C.POINTER(C.c_uint64))
        if self.lib.or_mc_set(_p32(a), a.shape[0], _p32(co), _p32(cl), co.shape[0], _p32(bs),
                              _p32(be), bs.shape[0], seed, s_begin, s_end, set_index, tp,
                              _p64(obs), _p64(k), C.byref(p), threads):
            raise ValueError("oracle rejected MC input")
        return totals, int(obs[0]), int(k[0]), p.value

    def mc_summary(self, totals, observed: int) -> dict:
        """Tally, middles and enrichment score of one MC test (Sec. "Monte Carlo
        Simulations", Fig. 3)."""
        t = np.ascontiguousarray(totals, np.uint64)
        ints = np.zeros(5, np.uint64)
        dbl = (C.c_double * 3)()
        tp = _p64(t) if t.size else C.cast(0, C.POINTER(C.c_uint64))
        if self.lib.or_mc_summary(tp, t.shape[0], observed, _p64(ints), dbl):
            raise ValueError("oracle: 64-bit overflow in the summary")
        return {"observed": int(ints[0]), "k_ge": int(ints[1]), "k_le": int(ints[2]),
                "median_lo": int(ints[3]), "median_hi": int(ints[4]), "p_enrich": dbl[0],
                "p_deplete": dbl[1], "log2_enrichment": dbl[2]}


_default: Oracle | None = None


def get() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default
