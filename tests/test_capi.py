"""The C-ABI library loads and exports every symbol include/bits.h declares.

No compute call here: these run without a GPU.  Argument checks that
return before touching CUDA are exercised too.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bits.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bits_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1208_3407_b300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1208_3407_b300 import build
        build.build()
    return _lib.load()


def test_header_lists_the_binding_exports():
    from paper_1208_3407_b300 import _lib
    assert _declared() == sorted(_lib.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_host_side_argument_checks(lib):
    from paper_1208_3407_b300 import _lib
    assert lib.bits_build_db(None, 0, None, None, None) == _lib.BITS_EINVAL
    h = C.c_void_p()
    assert lib.bits_build_db(None, 5, None, None, C.byref(h)) == _lib.BITS_EINVAL
    assert h.value is None
    assert lib.bits_build_db(C.c_void_p(256), 1 << 30, None, None, C.byref(h)) == _lib.BITS_EOVERFLOW
    assert lib.bits_build_db(C.c_void_p(260), 4, None, None, C.byref(h)) == _lib.BITS_EINVAL
    assert b"aligned" in lib.bits_last_error()
    bad = _lib.Opts(0, 0, 15, 0)
    assert lib.bits_build_db(C.c_void_p(256), 4, C.byref(bad), None, C.byref(h)) == _lib.BITS_EINVAL
    rmi_without_leaves = _lib.Opts(_lib.METHOD_RMI, 0, 0, 0)
    assert lib.bits_build_db(C.c_void_p(256), 4, C.byref(rmi_without_leaves), None,
                             C.byref(h)) == _lib.BITS_EINVAL
    assert lib.bits_count(None, None, 0, None, None, None) == _lib.BITS_EINVAL
    assert lib.bits_count_host(None, 1, None, 0, None, None, None) == _lib.BITS_EINVAL
    assert lib.bits_check(None, None) == _lib.BITS_EINVAL
    assert lib.bits_db_info(None, None, None, None, None) == _lib.BITS_EINVAL
    assert lib.bits_mc(None, 0, None, 0, None, None, 0, 0, 0, 0, None, None, None, None,
                       None) == _lib.BITS_EINVAL
    assert lib.bits_count_matrix(None, 1, None, None, 0, None, None) == _lib.BITS_EINVAL
    assert lib.bits_count_matrix_db(None, 1, None, 0, None, None) == _lib.BITS_EINVAL
    assert lib.bits_count_matrix_db(None, 0, None, 1, None, None) == _lib.BITS_EINVAL
    null2 = (C.c_void_p * 2)(None, None)
    assert lib.bits_count_matrix_db(null2, 2, null2, 2, None, None) == _lib.BITS_EINVAL
    assert lib.bits_count_matrix_db(None, 0, None, 0, None, None) == _lib.BITS_OK  # empty matrix
    unknown_flag = _lib.Opts(0, 0, 0, 2)
    assert lib.bits_build_db(C.c_void_p(256), 4, C.byref(unknown_flag), None,
                             C.byref(h)) == _lib.BITS_EINVAL
    # projection: size, mode and pointer checks
    assert lib.bits_project(None, None, None, 1 << 32, None, None, 0, 0, None, None,
                            None) == _lib.BITS_EOVERFLOW
    assert lib.bits_project(None, None, None, 0, None, None, 0, 2, None, None,
                            None) == _lib.BITS_EINVAL
    assert lib.bits_project(None, None, None, 3, None, None, 0, 0, None, None,
                            None) == _lib.BITS_EINVAL
    assert lib.bits_project(None, C.c_void_p(256), C.c_void_p(512), 3, None, None, 2, 0,
                            C.c_void_p(1024), None, None) == _lib.BITS_EINVAL   # ids missing
    assert lib.bits_project(None, None, None, 0, None, None, 0, 1, None, None, None) == _lib.BITS_OK
    # Monte-Carlo summary and screen
    assert lib.bits_mc_summary(None, 10, 0, None, None, None) == _lib.BITS_OK
    assert lib.bits_mc_summary(None, 10, 2, None, None, None) == _lib.BITS_EINVAL
    assert lib.bits_mc_summary(C.c_void_p(260), 10, 2, C.c_void_p(256), C.c_void_p(512),
                               None) == _lib.BITS_EINVAL                       # misaligned
    assert lib.bits_mc_matrix(None, 1, None, None, 1, None, None, 0, 0, 0, 0, None, None, None,
                              None) == _lib.BITS_EINVAL
    assert lib.bits_mc_matrix(None, 0, None, None, 0, None, None, 0, 0, 5, 4, None, None, None,
                              None) == _lib.BITS_EINVAL                       # end < begin
    assert lib.bits_mc_matrix(None, 0, None, None, 0, None, None, 0, 0, 0, 4, None, None, None,
                              None) == _lib.BITS_OK                           # nothing to do
    # enumeration
    assert lib.bits_enumerate_offsets(None, None, 0, None, None) == _lib.BITS_EINVAL
    assert lib.bits_enumerate_pairs(None, None, 0, None, None, None) == _lib.BITS_EINVAL
    # launch-parameter pins: validated on the host
    bad = _lib.Tuning(3, 0, 0, 0, 0)
    assert lib.bits_set_tuning(C.byref(bad)) == _lib.BITS_EINVAL
    bad = _lib.Tuning(-1, 0, 128, 512, 0)
    assert lib.bits_set_tuning(C.byref(bad)) == _lib.BITS_EINVAL
    good = _lib.Tuning(1, 256, 128, 2048, 16384)
    assert lib.bits_set_tuning(C.byref(good)) == _lib.BITS_OK
    got = _lib.Tuning()
    assert lib.bits_get_tuning(C.byref(got)) == _lib.BITS_OK
    assert (got.top_raise, got.block, got.mc_shuffles, got.mc_chunk, got.ap_chunk) == \
        (1, 256, 128, 2048, 16384)
    assert lib.bits_set_tuning(None) == _lib.BITS_OK
    assert lib.bits_get_tuning(C.byref(got)) == _lib.BITS_OK and got.top_raise == -1
    assert lib.bits_get_tuning(None) == _lib.BITS_EINVAL
    lib.bits_free(None)
    assert lib.bits_kernel_launches() == 0


def test_probe_library_exports_and_checks(lib):
    """The measurement probe lives in libbits_probe.so (include/bits_probe.h),
    outside the library's own C ABI; its argument checks return codes."""
    from paper_1208_3407_b300 import _lib, probe
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "bits_probe.h")).read(),
                  flags=re.S)
    declared = sorted(set(re.findall(r"\b(bits_[a-z_0-9]+)\s*\(", text)))
    assert declared == sorted(probe.EXPORTS)
    plib = probe.load()
    for name in declared:
        assert hasattr(plib, name), name
        assert not hasattr(lib, name), name            # not in the method's library
    rate = C.c_double()
    f = plib.bits_probe_random_reads
    assert f(None, 1 << 20, 1, 1, C.byref(rate), None) == _lib.BITS_EINVAL
    assert f(C.c_void_p(256), 100, 1, 1, C.byref(rate), None) == _lib.BITS_EINVAL
    assert f(C.c_void_p(256), 1 << 20, 0, 1, C.byref(rate), None) == _lib.BITS_EINVAL
    assert f(C.c_void_p(256), 1 << 20, 1, 0, C.byref(rate), None) == _lib.BITS_EINVAL
    assert f(C.c_void_p(256), 1 << 20, 1, 4, C.byref(rate), None) == _lib.BITS_EINVAL
    assert f(C.c_void_p(64), 1 << 20, 1, 2, C.byref(rate), None) == _lib.BITS_EINVAL
    assert f(C.c_void_p(64), 1 << 20, 1, 3, C.byref(rate), None) == _lib.BITS_EINVAL
    assert b"bits_probe_random_reads" in lib.bits_last_error()


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1208_3407_b300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        _lib.load()


def test_package_does_not_import_oracle():
    import sys
    import subprocess
    code = ("import sys, paper_1208_3407_b300, paper_1208_3407_b300._lib; "
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "False"
