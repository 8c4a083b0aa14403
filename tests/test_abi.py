"""The C ABI library loads and exports every symbol include/zk.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(zk_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2608_25203_b300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    from paper_2608_25203_b300 import zk
    assert declared_symbols() == set(zk.EXPORTS)


def test_host_only_entry_points(lib):
    lib.zk_version.restype = ctypes.c_char_p
    lib.zk_strerror.restype = ctypes.c_char_p
    lib.zk_strerror.argtypes = [ctypes.c_int]
    assert b"sm_103a" in lib.zk_version()
    assert lib.zk_strerror(1) == b"invalid argument"
    # argument validation happens before any CUDA call
    lib.zk_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
    c = ctypes.c_void_p()
    assert lib.zk_create(ctypes.byref(c), 48, 64, 1.0, 1.0, 1.0, 9.81, 3, 0) == 1
    assert lib.zk_create(ctypes.byref(c), 64, 64, 1.0, 1.0, 1.0, 9.81, 9, 0) == 1
    assert lib.zk_create(ctypes.byref(c), 64, 64, -1.0, 1.0, 1.0, 9.81, 3, 0) == 1
    assert not c.value


def test_no_oracle_import_in_product():
    pkg = os.path.join(ROOT, "paper_2608_25203_b300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "oracle" not in re.findall(r"(?:import|from)\s+(\w+)", txt), f
