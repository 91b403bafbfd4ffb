"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point that include/kcl.h declares.  No compute calls
(there is no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kcl.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kcl_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "kcl_build", os.path.join(ROOT, "paper_2203_13512_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("kcl_load_csr", "kcl_count", "kcl_list", "kcl_free_graph", "kcl_strerror",
                     "kcl_count_per_root", "kcl_stage_info"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (kcl_[a-z_0-9]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_names_statuses(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        getattr(lib, name)
    lib.kcl_strerror.restype = ctypes.c_char_p
    lib.kcl_strerror.argtypes = [ctypes.c_int]
    assert lib.kcl_strerror(0) == b"ok"
    assert b"invalid" in lib.kcl_strerror(1)
    assert lib.kcl_strerror(99) == b"unknown status"


def test_binding_mirrors_the_abi(lib_path):
    import paper_2203_13512_gb300 as kcl
    for name in _declared():
        assert hasattr(kcl, name), name


def test_arguments_rejected_without_touching_the_device(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.kcl_load_csr.restype = ctypes.c_int
    lib.kcl_load_csr.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                 ctypes.c_void_p, ctypes.c_void_p]
    assert lib.kcl_load_csr(0, None, None, 0, None, None) == 1
    lib.kcl_count.restype = ctypes.c_int
    lib.kcl_count.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p]
    c = ctypes.c_uint64()
    assert lib.kcl_count(None, 4, 0, ctypes.byref(c)) == 1
