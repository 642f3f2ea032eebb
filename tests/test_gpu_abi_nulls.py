"""Every entry point of the C ABI called with NULL handles and pointers (and
every size 1, which no call can honour with NULL data) returns an error status
(or, for the destroy calls, nothing) without touching memory.  The sweep runs
in a child process that names each call before making it, so a crash points at
the call."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SWEEP = r"""
import ctypes as C
import paper_2603_20336_b300 as gem
from paper_2603_20336_b300._abi import SIGNATURES
lib = gem.lib
skip = {"gem_version", "gem_device_check", "gem_last_error_message", "gem_kernel_launches"}
for name, (res, args) in SIGNATURES.items():
    if name in skip:
        continue
    vals = []
    for t in args:
        if t in (C.c_int32, C.c_int64, C.c_uint32, C.c_int, C.c_size_t, C.c_uint64):
            vals.append(1)
        else:
            vals.append(None)
    print("CALL", name, flush=True)
    rc = getattr(lib, name)(*vals)
    if res is None:
        print("OK", name, "void", flush=True)
    else:
        print("OK", name, int(rc), flush=True)
print("DONE", flush=True)
"""


def test_every_entry_point_rejects_null_arguments():
    r = subprocess.run([sys.executable, "-c", SWEEP], cwd=ROOT, capture_output=True, text=True, timeout=300)
    out = r.stdout.splitlines()
    assert r.returncode == 0 and out and out[-1] == "DONE", (
        "crashed at " + next((ln for ln in reversed(out) if ln.startswith("CALL")), "?") + "\n" + r.stderr[-2000:])
    bad = []
    for ln in out:
        if ln.startswith("OK"):
            _, name, rc = ln.split()
            if rc != "void" and int(rc) == 0:
                bad.append(name)
    assert not bad, f"returned GEM_OK on NULL arguments: {bad}"
