"""The C-ABI library builds for sm_103a, loads on a machine without a GPU, and
exports every entry point declared in include/*.h (no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(drts_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1611_08536_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_core_calls():
    names = declared_functions()
    for n in ["drts_assemble", "drts_step_n", "drts_inject_source", "drts_read_detectors",
              "drts_read_state", "drts_destroy", "drts_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1611_08536_gb300 import drts
    assert sorted(drts.SYMBOLS) == declared_functions()


def test_assemble_rejects_null_without_gpu(lib):
    lib.drts_assemble.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.drts_last_error.restype = ctypes.c_char_p
    lib.drts_last_error.argtypes = [ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert lib.drts_assemble(None, None, ctypes.byref(out)) == 1      # DRTS_EINVAL
    assert b"NULL" in lib.drts_last_error(None)


def test_host_allocation_failure_returns_status():
    """No C++ exception crosses the C ABI: drts_assemble with its address
    space capped below the host copy of the medium map (a 400^3 grid, 64 MB)
    returns DRTS_ENOMEM with a message instead of terminating the process.
    The copy is taken before any CUDA call, so this runs without a GPU."""
    import subprocess
    import sys
    code = r"""
import ctypes, resource
from paper_1611_08536_gb300 import drts, inputs as I
lib = drts.load()
prob = I.homogeneous(400, 0.1, (10.0, 0.01, 0.9, 1.4))
ps = drts.problem_struct(prob, 0)
h = ctypes.c_void_p()
vm = int(open("/proc/self/statm").read().split()[0]) * resource.getpagesize()
soft, hard = resource.getrlimit(resource.RLIMIT_AS)
resource.setrlimit(resource.RLIMIT_AS, (vm + (16 << 20), hard))
st = lib.drts_assemble(ctypes.byref(ps), None, ctypes.byref(h))
resource.setrlimit(resource.RLIMIT_AS, (soft, hard))
print(st, h.value is None, lib.drts_last_error(None).decode())
"""
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    st, null, msg = r.stdout.strip().split(" ", 2)
    assert int(st) == 2 and null == "True", r.stdout
    assert "drts_assemble" in msg and "host allocation failed" in msg, msg
