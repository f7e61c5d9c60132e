"""The bounds-checked build's index check, in a host build of the library header (no GPU, no
out-of-range device access): an index outside [0, n) returns false, is skipped, and the first
failure (site, index) is kept in the error word; the normal library reports the checked
entry point as unsupported."""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np

from paper_2607_00095_b300 import _abi

HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def lib():
    global _lib
    if _lib is None:
        out = os.path.join(tempfile.mkdtemp(), "libbounds_harness.so")
        subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-O2", "-std=c++17", "-DSNAP_BOUNDS_CHECK",
                               "-Xcompiler", "-fPIC", "-shared", "-o", out,
                               os.path.join(HERE, "csrc", "bounds_harness.cu")])
        L = C.CDLL(out)
        L.harness_check.argtypes = [C.POINTER(C.c_ulonglong), C.c_int, C.c_longlong, C.c_longlong]
        L.harness_checked_copy.argtypes = [C.c_void_p, C.c_void_p, C.c_longlong, C.c_longlong,
                                           C.c_longlong, C.POINTER(C.c_ulonglong)]
        _lib = L
    return _lib


def _word(site, i):
    return (site << 48) | (i & 0xFFFFFFFFFFFF)


def test_index_check_records_first_failure():
    L = lib()
    err = C.c_ulonglong(0)
    assert L.harness_check(C.byref(err), 3, 0, 10) == 1
    assert L.harness_check(C.byref(err), 3, 9, 10) == 1
    assert err.value == 0
    assert L.harness_check(C.byref(err), 3, 10, 10) == 0
    assert err.value == _word(3, 10)
    assert L.harness_check(C.byref(err), 5, -1, 10) == 0      # later failures keep the first
    assert err.value == _word(3, 10)
    err2 = C.c_ulonglong(0)
    assert L.harness_check(C.byref(err2), 4, -2, 10) == 0
    assert err2.value == _word(4, -2)


def test_checked_copy_skips_out_of_range_accesses():
    L = lib()
    n = 16
    src = np.arange(n + 8, dtype=np.float64)
    dst = np.full(n + 8, -1.0)
    err = C.c_ulonglong(0)
    done = L.harness_checked_copy(src.ctypes.data, dst.ctypes.data, n, 10, 10, C.byref(err))
    assert done == 6                                   # j = 10..15 copied, 16..19 skipped
    np.testing.assert_array_equal(dst[10:16], src[10:16])
    assert np.all(dst[16:] == -1.0) and np.all(dst[:10] == -1.0)
    assert err.value == _word(7, 16)


def test_normal_library_reports_checked_entry_unsupported():
    L = _abi.lib()
    w = C.c_ulonglong(123)
    assert L.snap_bounds_error(C.byref(w), 0) == 2
    assert w.value == 0
