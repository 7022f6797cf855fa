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


STRUCTS = [("Medium", "drts_medium"), ("ProblemC", "drts_problem"), ("Info", "drts_info"),
           ("TuneResult", "drts_tune_result"), ("ServerConfig", "drts_server_config"),
           ("RequestInfo", "drts_request_info"), ("ServerStats", "drts_server_stats"), ("FccInfo", "drts_fcc_info"),
           ("FccProblemC", "drts_fcc_problem")]


def test_binding_structs_match_header_layout(tmp_path):
    """Every ctypes structure of the binding has the C header's layout: the
    same field names at the same offsets with the same sizes, and the same
    total size (a C program compiled against include/drts.h prints them)."""
    import ctypes as C
    import shutil
    import subprocess
    from paper_1611_08536_gb300 import drts
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "drts.h"', "int main(void) {"]
    for py, c in STRUCTS:
        lines.append(f'printf("{py} sizeof %zu\\n", sizeof({c}));')
        for name, _ in getattr(drts, py)._fields_:
            lines.append(f'printf("{py} {name} %zu %zu\\n", offsetof({c}, {name}), sizeof((({c} *)0)->{name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for ln in filter(None, out):
        parts = ln.split()
        cls = getattr(drts, parts[0])
        if parts[1] == "sizeof":
            assert C.sizeof(cls) == int(parts[2]), parts
        else:
            f = getattr(cls, parts[1])
            assert (f.offset, f.size) == (int(parts[2]), int(parts[3])), parts
        seen += 1
    assert seen == sum(1 + len(getattr(drts, py)._fields_) for py, _ in STRUCTS)


def _prototypes():
    """(return type, name, [parameter declarations]) of every function the
    header declares."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "drts.h")).read(), flags=re.S)
    out = []
    for m in re.finditer(r"^([A-Za-z_][\w \*]*?)\b(drts_\w+)\s*\(([^)]*)\)\s*;", text, flags=re.M):
        params = [p.strip() for p in m.group(3).split(",") if p.strip() and p.strip() != "void"]
        out.append((m.group(1).strip(), m.group(2), params))
    return out


def test_binding_signatures_match_header():
    """The binding's argtypes follow each prototype: same number of
    parameters, the same scalar types, pointers where the header has them;
    char-pointer and void returns declared as such."""
    import ctypes as C
    from paper_1611_08536_gb300 import drts
    lib = drts.load()
    scalar = {"int32_t": C.c_int32, "int64_t": C.c_int64, "double": C.c_double}
    protos = _prototypes()
    assert len(protos) >= 30
    for ret, name, params in protos:
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == len(params), name
        for decl, t in zip(params, fn.argtypes):
            if "*" in decl:
                assert t in (C.c_void_p, C.c_char_p) or issubclass(t, C._Pointer), (name, decl, t)
            else:
                base = decl.split()[-2] if len(decl.split()) > 1 else decl
                if base.endswith("_fn"):           # callback typedefs: ctypes function pointers
                    assert issubclass(t, C._CFuncPtr), (name, decl, t)
                else:
                    assert t is scalar[base], (name, decl, t)
        if ret.replace(" ", "") == "constchar*":
            assert fn.restype is C.c_char_p, name
        elif ret == "void":
            assert fn.restype is None, name


def test_plain_c_program_uses_the_library(tmp_path):
    """A plain C11 program compiled against include/drts.h and linked with
    libdrts.so (no C++, no Python) calls the host-side entry points and gets
    the same stencil value as the binding; errors come back as statuses."""
    import shutil
    import subprocess
    import numpy as np
    from paper_1611_08536_gb300 import build, drts, inputs as I
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include <stdlib.h>
#include "drts.h"
int main(void) {
    drts_medium med = {10.0, 0.01, 0.9, 1.4};
    enum { N = 4 };
    uint8_t mov[N * N * N] = {0};
    drts_problem p = {0};
    p.nx = p.ny = p.nz = N; p.voxel_mm = 0.1; p.n_media = 1; p.media = &med;
    p.medium_of_voxel = mov; p.n_outside = 1.0; p.boundary = DRTS_FRESNEL;
    p.precision = DRTS_FP32; p.n_rhs = 1; p.det_face = DRTS_FACE_NONE;
    double *W = malloc(sizeof(double) * 26 * 27 * 26);
    drts_status st = drts_host_tables(&p, 0, W, NULL, NULL, NULL);
    /* direction +x is index 13; offset +x is (0+1)*9 + (0+1)*3 + 2 = 14 */
    printf("%d %.17g\n", (int)st, W[(13 * 27 + 14) * 26 + 13]);
    st = drts_host_tables(&p, 3, W, NULL, NULL, NULL);
    printf("%d %s\n", (int)st, drts_last_error(NULL));
    free(W);
    return 0;
}
''')
    exe = tmp_path / "use"
    libdir = os.path.dirname(lib)
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-ldrts", "-Wl,-rpath," + libdir, "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    st, val = out[0].split()
    prob = I.Problem((4, 4, 4), 0.1, [(10.0, 0.01, 0.9, 1.4)], np.zeros((4, 4, 4), np.uint8), 1.0,
                     I.FRESNEL, I.FP32, 1, -1, 1, 1, "c")
    W, _, _, _ = drts.host_tables(prob, 0)
    assert int(st) == 0 and float(val) == W[13, 14, 13]
    assert out[1].startswith(f"{drts.EINVAL} ") and "medium out of range" in out[1]


def test_alloc_fault_hook_needs_no_device():
    """The allocator fault is host state: arming and disarming it touches no
    device and always succeeds."""
    from paper_1611_08536_gb300 import build, drts
    build.build()
    lib = drts.load()
    assert lib.drts_set_alloc_fault(3) == drts.OK
    assert lib.drts_set_alloc_fault(-5) == drts.OK


def test_allocator_needs_both_functions():
    """drts_set_allocator takes both callbacks or neither (host state only)."""
    from paper_1611_08536_gb300 import build, drts
    build.build()
    lib = drts.load()
    keep = drts.ALLOC_FN(lambda n, s, u: None)
    assert lib.drts_set_allocator(keep, drts.FREE_FN(), None) == drts.EINVAL
    assert lib.drts_set_allocator(drts.ALLOC_FN(), drts.FREE_FN(), None) == drts.OK
