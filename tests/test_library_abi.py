"""The C-ABI library loads and exports every symbol include/nmg.h declares (no GPU calls)."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nmg.h")
LIB = os.path.join(ROOT, "paper_1904_02401_gb300", "libnmg.so")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nmg_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    if not os.path.exists(LIB):
        from paper_1904_02401_gb300 import build
        build.build()
    return LIB


def test_header_declares_the_boundary():
    names = declared()
    for required in ("nmg_create_hierarchy", "nmg_set_jacobian", "nmg_solve", "nmg_destroy_hierarchy",
                     "nmg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    import ctypes
    lib = ctypes.CDLL(lib_path)
    for name in declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (nmg_[a-z_0-9]+)", out))
    assert set(declared()) <= exported


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_1904_02401_gb300 import nmg
    assert set(declared()) <= set(nmg.EXPORTED)
    for name in declared():
        assert callable(getattr(nmg, name))
    assert nmg.nmg_last_error() == "no error"
