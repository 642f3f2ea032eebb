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


def test_store_file_validation_needs_no_gpu(lib, tmp_path):
    """gem_store_load checks a file's header, length, offsets and float values
    before it touches a device: a missing file, a foreign file, another version,
    a header whose sizes disagree with the file's length, bad offsets and a
    non-finite vector or centroid are refused with GEM_ERR_INVALID (1)."""
    import struct
    lib.gem_store_load.argtypes = [ctypes.c_char_p, ctypes.c_uint32, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_void_p)]
    lib.gem_store_load.restype = ctypes.c_int

    def load(path):
        out = ctypes.c_void_p()
        return lib.gem_store_load(str(path).encode(), 1, None, ctypes.byref(out)), out.value

    header = b"GEMSTORE" + struct.pack("<IIqqiiII", 1, 128, 2, 3, 0, 0, 0, 0)
    body = struct.pack("<3q", 0, 1, 3) + b"\0" * (3 * 128 * 4) + b"GEMEND01"
    cases = {
        "missing.gem": None,
        "foreign.gem": b"NOTASTORE" + b"\0" * 64,
        "version.gem": b"GEMSTORE" + struct.pack("<IIqqiiII", 2, 128, 2, 3, 0, 0, 0, 0) + body,
        "dim.gem": b"GEMSTORE" + struct.pack("<IIqqiiII", 1, 64, 2, 3, 0, 0, 0, 0) + body,
        "short.gem": header + body[:-9],
        "long.gem": header + body + b"x",
        "offsets.gem": header + struct.pack("<3q", 0, 2, 1) + body[24:],
        # finite-size files whose float arrays hold a NaN or an infinity: a NaN
        # centroid would make every dot NaN, so the file is refused before any
        # device work (the codes kernels also map NaN dots below every value)
        "nan_vector.gem": header + struct.pack("<3q", 0, 1, 3) + struct.pack("<f", float("nan"))
        + b"\0" * (3 * 128 * 4 - 4) + b"GEMEND01",
        "nan_centroid.gem": b"GEMSTORE" + struct.pack("<IIqqiiII", 1, 128, 2, 3, 1, 0, 0, 0)
        + struct.pack("<3q", 0, 1, 3) + b"\0" * (3 * 128 * 4) + struct.pack("<f", float("nan"))
        + b"\0" * (127 * 4) + b"GEMEND01",
        "inf_index_centroid.gem": b"GEMSTORE" + struct.pack("<IIqqiiII", 1, 128, 2, 3, 0, 1, 0, 0)
        + struct.pack("<3q", 0, 1, 3) + b"\0" * (3 * 128 * 4) + b"\0" * (127 * 4)
        + struct.pack("<f", float("inf")) + b"GEMEND01",
    }
    for name, data in cases.items():
        p = tmp_path / name
        if data is not None:
            p.write_bytes(data)
        code, handle = load(p)
        assert code == 1 and not handle, name
        if "nan" in name or "inf" in name:
            assert b"non-finite" in lib.gem_last_error_message(), name
    assert len(header) == 48
