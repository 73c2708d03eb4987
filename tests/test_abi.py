"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/mhd.h declares, and rejects bad arguments before it
touches a device (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_1804_03479_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "mhd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mhd_[a-zA-Z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_1804_03479_b300 import mhd
    return mhd.lib()


def test_every_declared_function_is_exported(lib):
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_1804_03479_b300 import mhd
    assert sorted(mhd.EXPORTS) == header_functions()


def test_init_rejects_bad_arguments_without_a_device(lib):
    from paper_1804_03479_b300 import mhd
    h = ctypes.c_void_p()
    g = mhd.Grid(0, 8, 8, 0.1)
    s = mhd.Scheme(0, 0, 0, 0, 0.3)
    assert lib.mhd_init(ctypes.byref(g), 5 / 3, ctypes.byref(s), None, ctypes.byref(h)) == mhd.MHD_EINVAL
    assert not h.value
    g = mhd.Grid(8, 8, 8, 0.1)
    assert lib.mhd_init(ctypes.byref(g), 1.0, ctypes.byref(s), None, ctypes.byref(h)) == mhd.MHD_EINVAL
    s = mhd.Scheme(1, 2, 0, 0, 0.3)   # CTU with primitive PLM is not built
    assert lib.mhd_init(ctypes.byref(g), 5 / 3, ctypes.byref(s), None, ctypes.byref(h)) == mhd.MHD_EUNSUPPORTED
    s = mhd.Scheme(0, 0, 7, 0, 0.3)
    assert lib.mhd_init(ctypes.byref(g), 5 / 3, ctypes.byref(s), None, ctypes.byref(h)) == mhd.MHD_EINVAL
    assert b"enum" in lib.mhd_last_error(None)


def test_null_context_calls_are_safe(lib):
    from paper_1804_03479_b300 import mhd
    assert lib.mhd_step(None, 0.1) == mhd.MHD_EINVAL
    assert lib.mhd_sync(None) == mhd.MHD_EINVAL
    lib.mhd_free(None)


def test_binding_return_types_match_header(lib):
    """the ctypes restype of every entry point is the header's return type"""
    src = open(os.path.join(ROOT, "include", "mhd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    want = {"mhd_status": ctypes.c_int, "int": ctypes.c_int, "long long": ctypes.c_longlong,
            "void": None, "const char*": ctypes.c_char_p}
    decls = re.findall(r"^(mhd_status|int|long long|void|const char\*)\s+(mhd_[a-zA-Z0-9_]+)\s*\(", src, flags=re.M)
    assert len(decls) == len(header_functions())
    for ret, name in decls:
        assert getattr(lib, name).restype == want[ret], (name, ret, getattr(lib, name).restype)
