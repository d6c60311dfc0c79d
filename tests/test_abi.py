"""The C-ABI library builds for sm_103a, loads, and exports every symbol the
header declares (no GPU needed: no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2304_10431_gb300 import _native
from paper_2304_10431_gb300 import build as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gslens.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(lens_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_core_api():
    names = declared_functions()
    for n in ["lens_plan_create", "lens_synthesis", "lens_adjoint", "lens_plan_destroy", "lens_plan_info",
              "lens_status_string", "lens_get_last_error", "lens_pointing"]:
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n), n
    # the binding declares exactly the header's functions
    assert sorted(_native.EXPORTS) == declared_functions()


def test_host_only_calls():
    lib = _native.load()
    assert lib.lens_nalm(4096, 4096) == 4097 * 4098 // 2
    assert lib.lens_nalm(10, 3) == 4 * (22 - 3) // 2
    assert lib.lens_nalm(3, 5) == 0
    assert lib.lens_status_string(0) == b"ok"
    assert lib.lens_version() >= 100
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    assert lib.lens_plan_create(ctypes.byref(h), -1, 0, 0, 0, None, None, None, 1e-5, 0, 0, None) == 1
    assert b"mmax" in lib.lens_last_error_message()
    assert lib.lens_get_last_error() == 1
    assert lib.lens_plan_create(ctypes.byref(h), 8, 8, 0, 0, None, None, None, 1e-8, 0, 0, None) == 3
    assert lib.lens_plan_create(ctypes.byref(h), 8, 8, 9, 0, None, None, None, 1e-5, 0, 0, None) == 1
    assert lib.lens_plan_create(ctypes.byref(h), 8, 8, 0, 10, None, None, None, 1e-5, 0, 0, None) == 1
    assert lib.lens_plan_create(ctypes.byref(h), 8, 8, 0, 0, None, None, None, 1e-14, 1, 0, None) == 3
    assert lib.lens_plan_destroy(None) == 0


def test_oracle_is_not_linked_into_the_product():
    src = " ".join(open(f).read() for f in B.sources())
    assert "oracle" not in src.lower()
    for f in os.listdir(os.path.dirname(B.__file__)):
        if f.endswith(".py"):
            assert "import oracle" not in open(os.path.join(os.path.dirname(B.__file__), f)).read()
