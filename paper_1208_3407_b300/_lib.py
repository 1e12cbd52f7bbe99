"""ctypes declarations of libbits_b300.so (the C ABI in include/bits.h).

Loading fails loudly when the compiled library is missing: there is no
Python or CPU fallback for any call.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbits_b300.so")

(BITS_OK, BITS_EINVAL, BITS_ENOMEM, BITS_ECUDA, BITS_EOVERFLOW, BITS_ETIMEOUT, BITS_ENOTIMPL,
 BITS_EINTERNAL) = range(8)
STATUS_NAMES = {0: "BITS_OK", 1: "BITS_EINVAL", 2: "BITS_ENOMEM", 3: "BITS_ECUDA",
                4: "BITS_EOVERFLOW", 5: "BITS_ETIMEOUT", 6: "BITS_ENOTIMPL", 7: "BITS_EINTERNAL"}

METHOD_AUTO, METHOD_SEARCH, METHOD_RMI, METHOD_MERGEPATH = range(4)

# Every symbol include/bits.h declares.
EXPORTS = ["bits_build_db", "bits_count", "bits_count_method", "bits_count_host", "bits_mc",
           "bits_count_matrix", "bits_count_matrix_db", "bits_db_info", "bits_check", "bits_free", "bits_last_error", "bits_kernel_launches",
           "bits_sort_intervals_noalloc", "bits_db_rmi", "bits_selftest_wait", "bits_project",
           "bits_mc_summary", "bits_mc_matrix", "bits_enumerate_offsets", "bits_enumerate_pairs",
           "bits_set_tuning", "bits_get_tuning"]


class BitsError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Opts(C.Structure):
    _fields_ = [("method", C.c_int32), ("rmi_leaves_log2", C.c_int32),
                ("top_tree_log2", C.c_int32), ("flags", C.c_int32)]


FLAG_ENUMERATE = 1


class Tuning(C.Structure):
    _fields_ = [("top_raise", C.c_int32), ("block", C.c_int32), ("mc_shuffles", C.c_int32),
                ("mc_chunk", C.c_int32), ("ap_chunk", C.c_int32)]


_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_1208_3407_b300.build` (nvcc, sm_103a)")
    lib = C.CDLL(LIB_PATH)
    vp, u32p, u64p = C.c_void_p, C.c_void_p, C.c_void_p
    st = C.c_int
    lib.bits_build_db.argtypes = [u32p, C.c_uint64, C.POINTER(Opts), vp, C.POINTER(C.c_void_p)]
    lib.bits_count.argtypes = [vp, u32p, C.c_uint64, u32p, u64p, vp]
    lib.bits_count_method.argtypes = [vp, C.c_int32, u32p, C.c_uint64, u32p, u64p, vp]
    lib.bits_count_host.argtypes = [vp, C.c_int32, vp, C.c_uint64, vp, vp, vp]
    lib.bits_mc.argtypes = [vp, C.c_int32, u32p, C.c_uint64, u32p, u32p, C.c_uint32, C.c_uint64,
                            C.c_uint32, C.c_uint32, u64p, C.POINTER(C.c_uint64),
                            C.POINTER(C.c_uint64), C.POINTER(C.c_double), vp]
    lib.bits_count_matrix.argtypes = [C.POINTER(C.c_void_p), C.c_uint32, C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_uint64), C.c_uint32, u64p, vp]
    lib.bits_count_matrix_db.argtypes = [C.POINTER(C.c_void_p), C.c_uint32,
                                         C.POINTER(C.c_void_p), C.c_uint32, u64p, vp]
    lib.bits_db_info.argtypes = [vp, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                 C.POINTER(C.c_uint64), C.POINTER(C.c_int32)]
    lib.bits_check.argtypes = [vp, vp]
    lib.bits_sort_intervals_noalloc.argtypes = [u32p, C.c_uint64, u32p, u32p, vp]
    lib.bits_selftest_wait.argtypes = [C.c_uint32, vp]
    lib.bits_set_tuning.argtypes = [C.POINTER(Tuning)]
    lib.bits_get_tuning.argtypes = [C.POINTER(Tuning)]
    lib.bits_enumerate_offsets.argtypes = [vp, u32p, C.c_uint64, u64p, vp]
    lib.bits_enumerate_pairs.argtypes = [vp, u32p, C.c_uint64, u64p, u32p, vp]
    lib.bits_mc_summary.argtypes = [u64p, C.c_uint32, C.c_uint32, u64p, vp, vp]
    lib.bits_mc_matrix.argtypes = [C.POINTER(C.c_void_p), C.c_uint32, C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_uint64), C.c_uint32, u32p, u32p, C.c_uint32,
                                   C.c_uint64, C.c_uint32, C.c_uint32, u64p, u64p, vp, vp]
    lib.bits_project.argtypes = [u32p, u32p, u32p, C.c_uint64, u32p, u32p, C.c_uint32, C.c_int32,
                                 u32p, u64p, vp]
    lib.bits_db_rmi.argtypes = [vp, C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_uint32),
                                C.POINTER(C.c_float), C.POINTER(C.c_float)]
    for f in ("bits_build_db", "bits_count", "bits_count_method", "bits_count_host", "bits_mc",
              "bits_count_matrix", "bits_count_matrix_db", "bits_db_info", "bits_check", "bits_sort_intervals_noalloc", "bits_db_rmi",
              "bits_selftest_wait", "bits_project", "bits_mc_summary", "bits_mc_matrix",
              "bits_enumerate_offsets", "bits_enumerate_pairs", "bits_set_tuning",
              "bits_get_tuning"):
        getattr(lib, f).restype = st
    lib.bits_free.argtypes = [vp]
    lib.bits_free.restype = None
    lib.bits_last_error.argtypes = []
    lib.bits_last_error.restype = C.c_char_p
    lib.bits_kernel_launches.argtypes = []
    lib.bits_kernel_launches.restype = C.c_uint64
    _lib = lib
    return lib


def check(status: int, where: str):
    if status != BITS_OK:
        msg = load().bits_last_error().decode(errors="replace")
        raise BitsError(status, where, msg)
