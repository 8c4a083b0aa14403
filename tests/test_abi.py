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


def test_binding_constants_match_header():
    """Every ZK_* constant the header defines (enum members and #defines) has the same value in
    the Python binding."""
    from paper_2608_25203_b300 import zk
    txt = "".join(open(os.path.join(ROOT, "include", f)).read()
                  for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    consts = {}
    for body in re.findall(r"enum\s*\{([^}]*)\}", txt):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            name, _, val = item.partition("=")
            nxt = int(val, 0) if val.strip() else nxt
            consts[name.strip()] = nxt
            nxt += 1
    for name, val in re.findall(r"#define\s+(ZK_[A-Z0-9_]+)\s+(-?\d+)\b", txt):
        consts[name] = int(val)
    consts = {k: v for k, v in consts.items() if k.startswith("ZK_")}
    assert {"ZK_RK4", "ZK_IFRK4", "ZK_IFAB2", "ZK_F32", "ZK_PAD_3"} <= set(consts)
    assert (consts["ZK_RK4"], consts["ZK_IFRK4"], consts["ZK_IFAB2"]) == (0, 1, 2)
    wrong = {k: (v, getattr(zk, k, None)) for k, v in consts.items() if getattr(zk, k, None) != v}
    assert not wrong, wrong


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
