"""Binary Interval Search (BITS) on one NVIDIA B300 -- Python binding.

A thin layer over the C ABI of ``libbits_b300.so`` (include/bits.h): it
checks tensor shapes and devices, passes raw pointers and the current torch
stream, and turns status codes into exceptions.  All computation runs in the
library's CUDA kernels; PyTorch only provides device memory and streams.

Interval sets are CUDA tensors of shape ``(n, 2)`` and dtype ``uint32`` (or
``int32`` holding the same bits), rows ``[start, end)`` on one genome-wide
coordinate line.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import (METHOD_AUTO, METHOD_MERGEPATH, METHOD_RMI, METHOD_SEARCH, BitsError,
                   LIB_PATH)

__all__ = ["Database", "count_matrix", "count_matrix_db", "project", "mc_summary", "mc_matrix", "McStats",
           "set_tuning", "get_tuning", "tuning",
           "kernel_launches", "BitsError", "METHOD_AUTO",
           "METHOD_SEARCH", "METHOD_RMI", "METHOD_MERGEPATH", "LIB_PATH", "device_view"]

_U32 = (torch.uint32, torch.int32)


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _intervals(x: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype not in _U32 or x.dim() != 2 or x.shape[1] != 2:
        raise TypeError(f"{name} must be a (n, 2) uint32/int32 tensor")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return x


def _u32_vec(x: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype not in _U32 or x.dim() != 1:
        raise TypeError(f"{name} must be a 1-D uint32/int32 CUDA tensor")
    return x.contiguous()


class _CAI:
    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


def device_view(ptr: int, n: int, dtype: str = "<u4") -> torch.Tensor:
    """A torch view of library-owned device memory (no copy)."""
    if n == 0:
        return torch.empty(0, dtype=torch.uint32, device="cuda")
    return torch.as_tensor(_CAI(ptr, n, dtype), device="cuda")


class Database:
    """A BITS database: the sorted start and end arrays of B (Algorithm 2)."""

    def __init__(self, b: torch.Tensor, *, method: int = 0, rmi_leaves_log2: int = 0,
                 top_tree_log2: int = 0, enumerate: bool = False, stream=None):
        b = _intervals(b, "b")
        self._lib = _lib.load()
        self.device = b.device
        opts = _lib.Opts(method, rmi_leaves_log2, top_tree_log2,
                         _lib.FLAG_ENUMERATE if enumerate else 0)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = self._lib.bits_build_db(b.data_ptr() if b.numel() else None, b.shape[0],
                                         C.byref(opts), _stream_ptr(stream), C.byref(h))
        _lib.check(st, "bits_build_db")
        self._h = h
        self.n = int(b.shape[0])
        bs, be, n, rmi = C.c_void_p(), C.c_void_p(), C.c_uint64(), C.c_int32()
        _lib.check(self._lib.bits_db_info(h, C.byref(bs), C.byref(be), C.byref(n), C.byref(rmi)),
                   "bits_db_info")
        self._bs, self._be, self.has_rmi = bs.value or 0, be.value or 0, bool(rmi.value)

    @property
    def handle(self) -> int:
        return self._h.value

    def sorted_arrays(self):
        """(B_S, B_E) as uint32 views of the database's own device memory."""
        return device_view(self._bs, self.n), device_view(self._be, self.n)

    def rmi(self, which: int = 0):
        """Learned index of the starts (0) or ends (1): (leaf table view, root slope, root icpt).

        The view is int32 [n_leaves, 8] over the database's own device memory:
        base_key, lo, slope bits, icpt bits, err_lo, err_hi, hi, reserved.
        """
        p, nl, ra, rb = C.c_void_p(), C.c_uint32(), C.c_float(), C.c_float()
        _lib.check(self._lib.bits_db_rmi(self._h, which, C.byref(p), C.byref(nl), C.byref(ra),
                                         C.byref(rb)), "bits_db_rmi")
        return device_view(p.value, nl.value * 8, "<i4").view(nl.value, 8), ra.value, rb.value

    def count(self, a: torch.Tensor, *, counts: bool | torch.Tensor = True, method: int | None = None,
              total: torch.Tensor | None = None, stream=None, check: bool = True):
        """Per-query counts (uint32, or None) and the uint64 total (1-element tensor)."""
        a = _intervals(a, "a")
        n = int(a.shape[0])
        if isinstance(counts, torch.Tensor):
            out = counts
            if out.dtype not in _U32 or out.numel() < n or not out.is_contiguous():
                raise TypeError("counts must be a contiguous uint32 tensor of >= n elements")
        else:
            out = torch.empty(n, dtype=torch.uint32, device=a.device) if counts else None
        if total is None:
            total = torch.empty(1, dtype=torch.uint64, device=a.device)
        sp = _stream_ptr(stream)
        cp = out.data_ptr() if (out is not None and n) else None
        ap = a.data_ptr() if n else None
        if method is None:
            st = self._lib.bits_count(self._h, ap, n, cp, total.data_ptr(), sp)
        else:
            st = self._lib.bits_count_method(self._h, method, ap, n, cp, total.data_ptr(), sp)
        _lib.check(st, "bits_count")
        if check:
            _lib.check(self._lib.bits_check(self._h, sp), "bits_count (device check)")
        return out, total

    def count_host(self, a, *, counts=True, total: torch.Tensor | None = None,
                   method: int = METHOD_AUTO, stream=None, check: bool = True):
        """bits_count_host: queries in host memory, counts and total back in it.

        ``a`` is a CPU tensor or numpy array of shape ``(n, 2)`` (uint32 or
        int32, C-contiguous).  ``counts`` is True (a new host array: page-
        locked when ``a`` is), False/None (total only) or a CPU uint32/int32
        tensor or numpy array of >= n elements that receives them.  ``total``
        is None (the total is returned as an int, which waits for it) or a
        page-locked uint64 CPU tensor of one element that receives it.
        Page-locked buffers are read and written in place by the search
        kernel; pageable ones are staged through device memory by the
        library.  With ``check`` the stream is synchronised and the device
        error word read (inverted queries raise); without it and with
        page-locked buffers the call is asynchronous and the results are in
        place once the stream has been synchronised.
        Returns ``(counts or None, total)``."""
        a_t = torch.from_numpy(a) if not isinstance(a, torch.Tensor) else a
        if a_t.is_cuda or a_t.dtype not in _U32 or a_t.dim() != 2 or a_t.shape[1] != 2:
            raise TypeError("a must be a host (n, 2) uint32/int32 array")
        if not a_t.is_contiguous():
            raise ValueError("a must be contiguous")
        n = int(a_t.shape[0])
        if counts is True:
            out = torch.empty(n, dtype=torch.uint32, pin_memory=bool(n) and a_t.is_pinned())
        elif counts is None or counts is False:
            out = None
        else:
            out = torch.from_numpy(counts) if not isinstance(counts, torch.Tensor) else counts
            if (out.is_cuda or out.dtype not in _U32 or out.numel() < n
                    or not out.is_contiguous()):
                raise TypeError("counts must be a contiguous host uint32 array of >= n elements")
        if total is None:
            tot = C.c_uint64()
            tp = C.addressof(tot)
        else:
            if total.is_cuda or total.dtype != torch.uint64 or total.numel() < 1:
                raise TypeError("total must be a host uint64 tensor of >= 1 element")
            tp = total.data_ptr()
        sp = _stream_ptr(stream)
        with torch.cuda.device(self.device):
            st = self._lib.bits_count_host(self._h, method, a_t.data_ptr() if n else None, n,
                                           out.data_ptr() if (out is not None and n) else None,
                                           tp, sp)
            _lib.check(st, "bits_count_host")
            if check:
                _lib.check(self._lib.bits_check(self._h, sp), "bits_count_host (device check)")
        return out, (tot.value if total is None else total)

    def enumerate(self, a: torch.Tensor, *, stream=None, check: bool = True):
        """Every intersecting pair (the enumeration problem of Sec. "Interval
        Set Intersection problem").

        Returns ``(offsets, pairs)``: uint64 offsets of shape ``(n + 1,)`` (query
        i's pairs are ``pairs[offsets[i]:offsets[i + 1]]``) and uint32 pairs of
        shape ``(total, 2)`` holding (query index, database index), each
        query's in descending database start order.  Needs a database built
        with ``enumerate=True``.  Reads the pair count back to size the output
        (one synchronisation)."""
        a = _intervals(a, "a")
        n = int(a.shape[0])
        sp = _stream_ptr(stream)
        off = torch.empty(n + 1, dtype=torch.uint64, device=a.device)
        ap = a.data_ptr() if n else None
        _lib.check(self._lib.bits_enumerate_offsets(self._h, ap, n, off.data_ptr(), sp),
                   "bits_enumerate_offsets")
        if stream is None:
            total = int(off[n].item())
        else:
            with torch.cuda.stream(stream):
                total = int(off[n].item())
        pairs = torch.empty((total, 2), dtype=torch.uint32, device=a.device)
        _lib.check(self._lib.bits_enumerate_pairs(self._h, ap, n, off.data_ptr(),
                                                  pairs.data_ptr() if total else None, sp),
                   "bits_enumerate_pairs")
        if check:
            _lib.check(self._lib.bits_check(self._h, sp), "bits_enumerate (device check)")
        return off, pairs

    def check(self, stream=None):
        _lib.check(self._lib.bits_check(self._h, _stream_ptr(stream)), "bits_check")

    def mc(self, a: torch.Tensor, contig_off: torch.Tensor, contig_len: torch.Tensor, *, seed: int,
           shuffle_begin: int = 0, shuffle_end: int, method: int = METHOD_AUTO,
           totals: torch.Tensor | None = None, stream=None):
        """Monte-Carlo test (Sec. "Monte Carlo Simulations"): (totals, observed,
        k_ge, p-value)."""
        a = _intervals(a, "a")
        co = _u32_vec(contig_off, "contig_off")
        cl = _u32_vec(contig_len, "contig_len")
        if co.numel() != cl.numel():
            raise ValueError("contig_off and contig_len differ in length")
        nsh = shuffle_end - shuffle_begin
        if totals is None:
            totals = torch.empty(max(nsh, 0), dtype=torch.uint64, device=a.device)
        obs, k, p = C.c_uint64(), C.c_uint64(), C.c_double()
        n = int(a.shape[0])
        st = self._lib.bits_mc(self._h, method, a.data_ptr() if n else None, n, co.data_ptr(),
                               cl.data_ptr(), co.numel(), seed, shuffle_begin, shuffle_end,
                               totals.data_ptr() if nsh > 0 else None, C.byref(obs), C.byref(k),
                               C.byref(p), _stream_ptr(stream))
        _lib.check(st, "bits_mc")
        return totals, obs.value, k.value, p.value

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.bits_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def count_matrix(dbs, a_sets, *, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """M[i][j] = total(A_i, B_j) for query sets A_i and databases B_j (uint64)."""
    lib = _lib.load()
    a_sets = [_intervals(a, f"a_sets[{i}]") for i, a in enumerate(a_sets)]
    n_db, n_sets = len(dbs), len(a_sets)
    dev = a_sets[0].device if a_sets else torch.device("cuda")
    if out is None:
        out = torch.empty((n_sets, n_db), dtype=torch.uint64, device=dev)
    hs = (C.c_void_p * max(1, n_db))(*[d._h.value for d in dbs])
    ps = (C.c_void_p * max(1, n_sets))(*[a.data_ptr() if a.shape[0] else None for a in a_sets])
    ns = (C.c_uint64 * max(1, n_sets))(*[int(a.shape[0]) for a in a_sets])
    st = lib.bits_count_matrix(hs, n_db, ps, ns, n_sets, out.data_ptr() if out.numel() else None,
                               _stream_ptr(stream))
    _lib.check(st, "bits_count_matrix")
    return out


def count_matrix_db(a_dbs, b_dbs, *, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """M[i][j] = total(A_i, B_j) with the query sets given as databases too
    (bits_count_matrix_db): each pair is counted from its smaller side's
    sorted keys in its larger side's tree."""
    lib = _lib.load()
    n_a, n_b = len(a_dbs), len(b_dbs)
    dev = (a_dbs or b_dbs)[0].device if (a_dbs or b_dbs) else torch.device("cuda")
    if out is None:
        out = torch.empty((n_a, n_b), dtype=torch.uint64, device=dev)
    if out.dtype != torch.uint64 or tuple(out.shape) != (n_a, n_b) or not out.is_contiguous():
        raise TypeError("out must be a contiguous uint64 tensor of shape (len(a_dbs), len(b_dbs))")
    ha = (C.c_void_p * max(1, n_a))(*[d._h.value for d in a_dbs])
    hb = (C.c_void_p * max(1, n_b))(*[d._h.value for d in b_dbs])
    st = lib.bits_count_matrix_db(ha, n_a, hb, n_b, out.data_ptr() if out.numel() else None,
                                  _stream_ptr(stream))
    _lib.check(st, "bits_count_matrix_db")
    return out


def project(start: torch.Tensor, end: torch.Tensor, *, contig: torch.Tensor | None = None,
            contig_off: torch.Tensor | None = None, contig_len: torch.Tensor | None = None,
            closed: bool = False, out: torch.Tensor | None = None, stream=None):
    """Map chromosome-local (optionally closed) intervals onto the half-open
    genome-wide line (Sec. "BITS Algorithm" (projection)).  Returns
    ``(intervals (n, 2) uint32, n_rejected)`` where ``n_rejected`` is a
    1-element uint64 device tensor; rejected rows are ``(2^32 - 1, 0)``.
    Without a contig table the line is one contig at 0."""
    lib = _lib.load()
    s = _u32_vec(start, "start")
    e = _u32_vec(end, "end")
    n = int(s.numel())
    if e.numel() != n:
        raise ValueError("start and end differ in length")
    nc = 0
    cp = op = lp = None
    if contig_off is not None or contig_len is not None or contig is not None:
        if contig is None or contig_off is None or contig_len is None:
            raise ValueError("contig, contig_off and contig_len go together")
        c = _u32_vec(contig, "contig")
        co = _u32_vec(contig_off, "contig_off")
        cl = _u32_vec(contig_len, "contig_len")
        if c.numel() != n or co.numel() != cl.numel():
            raise ValueError("contig ids or contig table have the wrong length")
        nc = int(co.numel())
        cp = c.data_ptr() if n else None
        op, lp = co.data_ptr(), cl.data_ptr()
    if out is None:
        out = torch.empty((n, 2), dtype=torch.uint32, device=s.device)
    else:
        out = _intervals(out, "out")
        if out.shape[0] != n:
            raise ValueError("out has the wrong number of rows")
    rej = torch.empty(1, dtype=torch.uint64, device=s.device)
    st = lib.bits_project(cp, s.data_ptr() if n else None, e.data_ptr() if n else None, n, op, lp,
                          nc, 1 if closed else 0, out.data_ptr() if n else None, rej.data_ptr(),
                          _stream_ptr(stream))
    _lib.check(st, "bits_project")
    return out, rej


class McStats:
    """Device array of bits_mc_stat records (include/bits.h), 64 bytes each.

    ``raw`` is a uint64 tensor of shape ``shape + (8,)``; the fields are views
    of it: observed, k_ge, k_le, median_lo, median_hi (uint64) and p_enrich,
    p_deplete, log2_enrichment (float64)."""

    INTS = ("observed", "k_ge", "k_le", "median_lo", "median_hi")
    DBLS = ("p_enrich", "p_deplete", "log2_enrichment")

    def __init__(self, raw: torch.Tensor):
        self.raw = raw

    def __getattr__(self, name):
        if name in McStats.INTS:
            return self.raw[..., McStats.INTS.index(name)]
        if name in McStats.DBLS:
            return self.raw[..., 5 + McStats.DBLS.index(name)].view(torch.float64)
        raise AttributeError(name)

    def to_dicts(self):
        """Host copies, one dict per test (row-major order)."""
        h = self.raw.reshape(-1, 8).cpu()
        ints = h[:, :5].tolist()
        dbl = h[:, 5:].contiguous().view(torch.float64).tolist()
        return [dict(zip(McStats.INTS + McStats.DBLS, [int(x) for x in i] + d))
                for i, d in zip(ints, dbl)]


def _u64(x: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype not in (torch.uint64, torch.int64):
        raise TypeError(f"{name} must be a uint64/int64 CUDA tensor")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return x


def mc_summary(totals: torch.Tensor, observed: torch.Tensor, *, stream=None) -> McStats:
    """Tallies, middle totals, p-values and Fig. 3 score of Monte-Carlo tests.

    ``totals`` has shape ``(..., N)`` (one row of shuffled totals per test) and
    ``observed`` the leading shape ``(...)``."""
    lib = _lib.load()
    totals = _u64(totals, "totals")
    observed = _u64(observed, "observed")
    shape = tuple(totals.shape[:-1])
    if tuple(observed.shape) != shape:
        raise ValueError("observed must have the shape of totals without its last axis")
    n_tests = int(observed.numel())
    n_sh = int(totals.shape[-1])
    raw = torch.empty(shape + (8,), dtype=torch.uint64, device=totals.device)
    st = lib.bits_mc_summary(totals.data_ptr() if totals.numel() else None, n_sh, n_tests,
                             observed.data_ptr() if n_tests else None,
                             raw.data_ptr() if n_tests else None, _stream_ptr(stream))
    _lib.check(st, "bits_mc_summary")
    return McStats(raw)


def mc_matrix(dbs, a_sets, contig_off: torch.Tensor, contig_len: torch.Tensor, *, seed: int,
              shuffle_begin: int = 0, shuffle_end: int, stats: bool = True, out=None, stream=None):
    """Monte-Carlo screen (Sec. "Novel genomic relationships"): (observed
    [S, D], totals [S, D, N], McStats or None).

    ``out`` may pass the three output tensors (observed, totals, raw stats or
    None) to reuse; the launch graph is cached per output address."""
    lib = _lib.load()
    a_sets = [_intervals(a, f"a_sets[{i}]") for i, a in enumerate(a_sets)]
    co = _u32_vec(contig_off, "contig_off")
    cl = _u32_vec(contig_len, "contig_len")
    if co.numel() != cl.numel():
        raise ValueError("contig_off and contig_len differ in length")
    n_db, n_sets = len(dbs), len(a_sets)
    nsh = shuffle_end - shuffle_begin
    if nsh < 0:
        raise ValueError("shuffle_end < shuffle_begin")
    dev = a_sets[0].device if a_sets else torch.device("cuda")
    if out is not None:
        observed, totals, raw = out
        if tuple(observed.shape) != (n_sets, n_db) or tuple(totals.shape) != (n_sets, n_db, nsh) \
                or (raw is not None and tuple(raw.shape) != (n_sets, n_db, 8)):
            raise ValueError("out tensors have the wrong shapes")
        for t, nm in ((observed, "observed"), (totals, "totals")):
            _u64(t, nm)
        if raw is not None:
            _u64(raw, "stats")
    else:
        observed = torch.empty((n_sets, n_db), dtype=torch.uint64, device=dev)
        totals = torch.empty((n_sets, n_db, nsh), dtype=torch.uint64, device=dev)
        raw = torch.empty((n_sets, n_db, 8), dtype=torch.uint64, device=dev) if stats else None
    hs = (C.c_void_p * max(1, n_db))(*[d._h.value for d in dbs])
    ps = (C.c_void_p * max(1, n_sets))(*[a.data_ptr() if a.shape[0] else None for a in a_sets])
    ns = (C.c_uint64 * max(1, n_sets))(*[int(a.shape[0]) for a in a_sets])
    st = lib.bits_mc_matrix(hs, n_db, ps, ns, n_sets, co.data_ptr(), cl.data_ptr(), co.numel(),
                            seed, shuffle_begin, shuffle_end,
                            observed.data_ptr() if observed.numel() else None,
                            totals.data_ptr() if totals.numel() else None,
                            raw.data_ptr() if (raw is not None and raw.numel()) else None,
                            _stream_ptr(stream))
    _lib.check(st, "bits_mc_matrix")
    return observed, totals, (McStats(raw) if raw is not None else None)


def set_tuning(top_raise: int = -1, block: int = 0, mc_shuffles: int = 0, mc_chunk: int = 0,
               ap_chunk: int = 0) -> None:
    """Pin launch parameters for later calls on this thread (bits_set_tuning);
    the defaults unpin (the autotuner decides)."""
    t = _lib.Tuning(top_raise, block, mc_shuffles, mc_chunk, ap_chunk)
    _lib.check(_lib.load().bits_set_tuning(C.byref(t)), "bits_set_tuning")


def get_tuning() -> dict:
    """The parameters pinned on this thread (-1 / 0: tuned)."""
    t = _lib.Tuning()
    _lib.check(_lib.load().bits_get_tuning(C.byref(t)), "bits_get_tuning")
    return {f: getattr(t, f) for f, _ in _lib.Tuning._fields_}


class tuning:
    """Context manager: pin launch parameters inside a ``with`` block."""

    def __init__(self, **kw):
        self.kw = kw

    def __enter__(self):
        self.prev = get_tuning()
        set_tuning(**self.kw)
        return self

    def __exit__(self, *exc):
        set_tuning(**self.prev)
        return False


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(_lib.load().bits_kernel_launches())
