"""The C ABI library builds for sm_103a, loads, and exports every function
include/hap.h declares (no GPU work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(hap_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1403_7394_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("hap_create", "hap_set_similarity", "hap_build_similarity", "hap_iterate",
                     "hap_exemplars", "hap_net_similarity", "hap_get_state", "hap_set_state", "hap_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(libpath):
    lib = ctypes.CDLL(libpath)
    lib.hap_strerror.restype = ctypes.c_char_p
    assert lib.hap_strerror(0) == b"HAP_OK"
    assert b"invalid" in lib.hap_strerror(-1)
    assert lib.hap_create(2, 1, None, ctypes.c_float(0.5), None, None, 0, None) == -1  # out == NULL
    assert lib.hap_iterate(None, 1) == -1
    assert lib.hap_sync(None) == -1
    assert lib.hap_band_create(ctypes.c_int64(2), ctypes.c_int64(0), ctypes.c_int64(1), 1, None, ctypes.c_float(0.5),
                               None, None) == -1  # out == NULL
    assert lib.hap_band_rows(None, None) == -1
    assert lib.hap_band_columns(None, None, 1, None) == -1
