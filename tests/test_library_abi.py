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
    assert isinstance(nmg.nmg_last_error(), str)   # never NULL (earlier tests may have set a message)


def _declared_arities():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(nmg_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        name, args = m.group(1), m.group(2).strip()
        if name in out:
            continue
        out[name] = 0 if args in ("", "void") else len(args.split(","))
    return out


def test_binding_argument_counts_match_header(lib_path):
    from paper_1904_02401_gb300 import nmg
    arity = _declared_arities()
    assert set(arity) == set(declared())
    for name, n in arity.items():
        f = getattr(nmg._lib, name)
        assert len(f.argtypes) == n, (name, len(f.argtypes), n)


def test_invalid_arguments_refused_before_the_device(lib_path):
    """Host-side checks of the multi-vector and batching entry points: NULL
    handles, column counts and batch widths out of range return
    NMG_ERR_INVALID without a CUDA call (this runs without a GPU)."""
    import numpy as np

    from paper_1904_02401_gb300 import nmg
    o = nmg.nmg_solve_opts()
    assert nmg.nmg_default_opts(o) == nmg.NMG_OK
    buf = np.zeros(4)
    assert nmg.nmg_vcycle_many(None, o, 1, buf, buf) == nmg.NMG_ERR_INVALID
    assert nmg.nmg_solve_many(None, 1, buf, buf, o) == nmg.NMG_ERR_INVALID
    assert nmg.nmg_server_set_batching(None, 8) == nmg.NMG_ERR_INVALID
    assert nmg.nmg_server_set_workspaces(None, 1) == nmg.NMG_ERR_INVALID
    assert nmg.nmg_server_memory(None, None, None) == nmg.NMG_ERR_INVALID
    assert nmg.nmg_set_wait_limit(None, 1) == nmg.NMG_ERR_INVALID
    assert "NULL" in nmg.nmg_last_error() or "bad server" in nmg.nmg_last_error()
