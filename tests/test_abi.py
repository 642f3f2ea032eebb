"""The C-ABI library loads and exports every symbol include/gem.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2603_20336_b300", "libgem.so")


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(gem_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    return ctypes.CDLL(LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2603_20336_b300 import _abi
    assert set(_abi.SIGNATURES) == _declared()


def test_host_side_errors_without_gpu(lib):
    from paper_2603_20336_b300 import _abi
    _abi.declare(lib)
    assert lib.gem_version() >= 100
    out = ctypes.c_void_p()
    # NULL inputs are rejected before any device work
    assert lib.gem_store_create(None, None, 10, 128, 3, 1, None, ctypes.byref(out)) == 1
    assert b"NULL" in lib.gem_last_error_message()
    assert lib.gem_workspace_create(None, 1, 1, 1, 0, 0, ctypes.byref(out)) == 1
    assert lib.gem_topk(None, None, None, 1, 1, None, 1, None, None, None) == 1
