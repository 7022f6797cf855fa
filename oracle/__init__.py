"""FP64 CPU oracle of the DRTS time step (arXiv:1611.08536, Eq. 18-27).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product (the
CUDA library and its binding) never does, and shares no code with it.

The arithmetic lives in ``drts_oracle.c`` (plain C, FP64, no FMA
contraction); this module only compiles it with gcc and marshals numpy arrays.

Parity status of each function (pins are in ``tests/test_oracle_pins.py``):
  * ``raw_stencil``   pinned: closed-form weights of Eq. 18/19, HG g=0, Eq. 24
                      column sums; the HG kernel's mean cosine slope (Legendre
                      expansion), its g -> -g reflection and forward limit;
                      the quadrature-weighted kernel (problem field
                      ``direction_weights``) by its weights' sphere averages
                      up to degree 7, its mean cosine and the cube's 48
                      symmetries.
  * ``assemble``      pinned: column sums, mirror conservation, dense brute
                      force on 4^3, ballistic translation, single-scatter line,
                      irreducibility, invariance under the cube's symmetries
                      (tests/test_oracle_symmetry.py).
  * ``column_info``   pinned: Fresnel normal incidence, total internal
                      reflection, ledger closure.
  * ``run``           pinned: conservation, pure decay, dense matrix powers;
                      sparse detector rows against the face detector, the
                      state itself and the ledger.
  * ``sensor_response`` pinned: delta response, box window vs a library
                      convolution, linearity.
  * ``source_column`` pinned: closed-form axis-direction split (1 - f, f),
                      column sums exp(-mu_a f L), f -> 0 Dirac, f = 1 equals
                      A's column, mirror conservation.
  * interface / edge folding geometry (Section 4.2 readings): parity
    unpinned beyond the invariants above; the paper prints no numbers for it.

``oracle.fcc`` (numpy) is the same step on the close-packed sphere partition
of Section 3; its pins are in ``tests/test_oracle_fcc.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "drts_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OPEN, MIRROR, FRESNEL = 0, 1, 2
NDIR = 26


def build(force: bool = False, plant: str | None = None) -> str:
    """Compile the oracle with gcc (OpenMP when available).  ``plant`` names a
    planted mistake (PLANT_* in drts_oracle.c) for the pin self-test; it is
    built into a separate library and never used otherwise."""
    os.makedirs(_BUILD, exist_ok=True)
    lib = _LIB if plant is None else os.path.join(_BUILD, f"liboracle_{plant}.so")
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(_SRC)):
        return lib
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11",
            _SRC, "-o", lib + ".tmp", "-lm"]
    if plant is not None:
        base.insert(1, f"-D{plant}")
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(lib + ".tmp", lib)
    return lib


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("h", ctypes.c_double),
        ("n_media", ctypes.c_int32),
        ("mu_s", ctypes.c_void_p), ("mu_a", ctypes.c_void_p),
        ("g", ctypes.c_void_p), ("n", ctypes.c_void_p),
        ("medium", ctypes.c_void_p),
        ("n_outside", ctypes.c_double),
        ("boundary", ctypes.c_int32),
        ("det_face", ctypes.c_int32),
        ("det_nu", ctypes.c_int32), ("det_nv", ctypes.c_int32),
        ("interface", ctypes.c_int32),
        ("direction_weights", ctypes.c_int32),
    ]


def _bind(path):
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER(_Problem)
    vp = ctypes.c_void_p
    lib.orc_assemble.restype = vp
    lib.orc_assemble.argtypes = [P, ctypes.c_int, ctypes.c_int]
    lib.orc_csr_info.argtypes = [vp, vp, vp, vp]
    lib.orc_csr_copy.argtypes = [vp, vp, vp, vp]
    lib.orc_csr_free.argtypes = [vp]
    lib.orc_column_info.argtypes = [P, vp, vp, vp, vp]
    lib.orc_spmv.argtypes = [vp, vp, vp, ctypes.c_int]
    lib.orc_run.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int64,
                            ctypes.c_int32, vp, vp, ctypes.c_int64,
                            ctypes.c_int32, vp, vp, vp, vp, vp,
                            ctypes.c_int32, vp, vp,
                            ctypes.c_int64, vp, vp, vp, ctypes.c_int32, vp,
                            ctypes.c_int]
    lib.orc_sensor_response.argtypes = [vp, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.c_int32, vp, vp]
    lib.orc_source_column.restype = ctypes.c_int
    lib.orc_source_column.argtypes = [P, ctypes.c_int64, ctypes.c_double,
                                      ctypes.c_int32, vp, vp, vp]
    lib.orc_raw_stencil.argtypes = [P, ctypes.c_int, vp]
    lib.orc_two_step_stencil.argtypes = [P, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    lib.orc_fresnel.restype = ctypes.c_double
    lib.orc_fresnel.argtypes = [ctypes.c_double] * 3
    lib.orc_direction.argtypes = [ctypes.c_int, vp]
    return lib


class planted:
    """Context manager: route the module's functions to an oracle built with
    one planted mistake (pin self-test only)."""

    def __init__(self, name):
        self.name = name

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        _lib = _bind(build(plant=self.name))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Problem:
    """Marshals a problem description (any object with the fields of
    ``paper_1611_08536_gb300.inputs.Problem``) into the oracle's struct."""

    def __init__(self, prob):
        self.keep = [
            np.ascontiguousarray([m[0] for m in prob.media], dtype=np.float64),
            np.ascontiguousarray([m[1] for m in prob.media], dtype=np.float64),
            np.ascontiguousarray([m[2] for m in prob.media], dtype=np.float64),
            np.ascontiguousarray([m[3] for m in prob.media], dtype=np.float64),
            np.ascontiguousarray(prob.medium_of_voxel, dtype=np.uint8).ravel(),
        ]
        nx, ny, nz = prob.shape
        assert self.keep[4].size == nx * ny * nz
        self.s = _Problem(nx, ny, nz, float(prob.voxel_mm), len(prob.media),
                          _ptr(self.keep[0]), _ptr(self.keep[1]),
                          _ptr(self.keep[2]), _ptr(self.keep[3]),
                          _ptr(self.keep[4]), float(prob.n_outside),
                          int(prob.boundary), int(prob.det_face),
                          int(prob.det_nu), int(prob.det_nv),
                          int(getattr(prob, "interface", 0)),
                          int(getattr(prob, "direction_weights", 0)))
        self.shape = (nx, ny, nz)
        self.n_states = nx * ny * nz * NDIR


class CSR:
    """Oracle CSR rows (canonical row order, ascending columns)."""

    def __init__(self, row_ptr, col, val, row0):
        self.row_ptr, self.col, self.val, self.row0 = row_ptr, col, val, row0
        self._h = None

    @property
    def n_rows(self):
        return self.row_ptr.size - 1

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def __del__(self):
        if self._h is not None and _lib is not None:
            _lib.orc_csr_free(self._h)
            self._h = None


def assemble(prob, z0: int = 0, z1: int | None = None) -> CSR:
    """Rows of A (Eq. 21-23) for voxel planes [z0, z1)."""
    lib = _load()
    P = prob if isinstance(prob, Problem) else Problem(prob)
    if z1 is None:
        z1 = P.shape[2]
    h = lib.orc_assemble(ctypes.byref(P.s), int(z0), int(z1))
    if not h:
        raise ValueError("oracle: invalid problem or plane range")
    n_rows, nnz, row0 = (np.zeros(1, np.int64) for _ in range(3))
    lib.orc_csr_info(h, _ptr(n_rows), _ptr(nnz), _ptr(row0))
    rp = np.empty(int(n_rows[0]) + 1, np.int64)
    col = np.empty(int(nnz[0]), np.int32)
    val = np.empty(int(nnz[0]), np.float64)
    lib.orc_csr_copy(h, _ptr(rp), _ptr(col), _ptr(val))
    c = CSR(rp, col, val, int(row0[0]))
    c._h = h
    return c


def column_info(prob):
    """Per-state absorb, exit_total, exit_det and detector patch (Eq. 8, 27)."""
    lib = _load()
    P = prob if isinstance(prob, Problem) else Problem(prob)
    n = P.n_states
    ab, ex, ed = (np.empty(n, np.float64) for _ in range(3))
    patch = np.empty(n, np.int32)
    if lib.orc_column_info(ctypes.byref(P.s), _ptr(ab), _ptr(ex), _ptr(ed),
                           _ptr(patch)):
        raise ValueError("oracle: invalid problem")
    return ab, ex, ed, patch


def spmv(csr: CSR, x: np.ndarray, n_threads: int = 0) -> np.ndarray:
    """y = A x over the rows of ``csr`` (x in canonical state order)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(csr.n_rows, np.float64)
    if csr._h is None:
        raise ValueError("CSR not owned by the oracle")
    lib.orc_spmv(csr._h, _ptr(x), _ptr(y), int(n_threads))
    return y


def run(prob, csr: CSR, n_steps: int, sources, x0=None, t_begin: int = 0,
        colinfo=None, n_threads: int = 0, point=None):
    """Run Eq. 26 for ``n_steps`` from ``x0`` (zeros by default).

    ``sources`` = (state_idx int64[], weight float64[], t0, profile float64[]).
    Returns (x, det[n_steps][n_patch], ledger[4] = {sum x, injected,
    absorbed, exited}).  With ``point`` = (n_det, det int32[], state int64[],
    weight float64[]) (sparse detector rows F of Eq. 27) a fourth item,
    pdet[n_steps][n_det], is returned.
    """
    lib = _load()
    P = prob if isinstance(prob, Problem) else Problem(prob)
    if csr.row0 != 0 or csr.n_rows != P.n_states:
        raise ValueError("run needs the full-grid CSR")
    ab, ex, ed, patch = colinfo if colinfo is not None else column_info(P)
    x = (np.zeros(P.n_states) if x0 is None
         else np.array(x0, dtype=np.float64, copy=True))
    st, w, t0, prof = sources
    st = np.ascontiguousarray(st, dtype=np.int64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    prof = np.ascontiguousarray(prof, dtype=np.float64)
    n_patch = max(int(patch.max()) + 1, 1)
    det = np.zeros((n_steps, n_patch), np.float64)
    ledger = np.zeros(4, np.float64)
    if point is not None:
        n_fdet = int(point[0])
        fd = np.ascontiguousarray(point[1], dtype=np.int32)
        fs = np.ascontiguousarray(point[2], dtype=np.int64)
        fw = np.ascontiguousarray(point[3], dtype=np.float64)
        pdet = np.zeros((n_steps, max(n_fdet, 1)), np.float64)
        fargs = (fd.size, _ptr(fd), _ptr(fs), _ptr(fw), n_fdet, _ptr(pdet))
    else:
        fargs = (0, None, None, None, 0, None)
    rc = lib.orc_run(csr._h, _ptr(x), int(t_begin), int(n_steps), st.size,
                     _ptr(st), _ptr(w), int(t0), prof.size, _ptr(prof),
                     _ptr(ab), _ptr(ex), _ptr(ed), _ptr(patch), n_patch,
                     _ptr(det), _ptr(ledger), *fargs, int(n_threads))
    if rc:
        raise RuntimeError(f"oracle run failed ({rc})")
    if point is not None:
        return x, det, ledger, pdet[:, :n_fdet]
    return x, det, ledger


def sensor_response(D, w: int, h):
    """Eq. 27 sensor output M[t][d] = sum_{|t-k| <= w} h[t-k+w] D[k][d]."""
    lib = _load()
    D = np.ascontiguousarray(D, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    if D.ndim != 2 or h.size != 2 * w + 1:
        raise ValueError("D must be [T][n_det] and h must have 2w+1 taps")
    M = np.empty_like(D)
    lib.orc_sensor_response(_ptr(D), D.shape[0], D.shape[1], int(w), _ptr(h), _ptr(M))
    return M


def source_column(prob, state: int, frac: float, cap: int = 4096):
    """States and values reached at the end of a step by a unit population
    emitted from ``state`` after the fraction 1 - ``frac`` of the step
    (Section 4.1 / Eq. 26 source partition).  Returns (states, values,
    exit_mass)."""
    lib = _load()
    P = prob if isinstance(prob, Problem) else Problem(prob)
    out_s = np.empty(cap, np.int64)
    out_w = np.empty(cap, np.float64)
    ex = np.zeros(1, np.float64)
    cnt = lib.orc_source_column(ctypes.byref(P.s), int(state), float(frac), int(cap),
                                _ptr(out_s), _ptr(out_w), _ptr(ex))
    if cnt < 0:
        raise ValueError(f"oracle: source_column failed ({cnt})")
    return out_s[:cnt].copy(), out_w[:cnt].copy(), float(ex[0])


def raw_stencil(prob, k: int) -> np.ndarray:
    """Unfolded W[n][o][m] of medium k, o = (oz+1)*9 + (oy+1)*3 + (ox+1)."""
    lib = _load()
    P = prob if isinstance(prob, Problem) else Problem(prob)
    W = np.empty((NDIR, 27, NDIR), np.float64)
    if lib.orc_raw_stencil(ctypes.byref(P.s), int(k), _ptr(W)):
        raise ValueError("oracle: invalid problem")
    return W


def two_step_stencil(prob, k1: int, k2: int):
    """Two-step entries of a source in medium k1 next to a z layer of medium
    k2: (S1, S0, active) with S1/S0[n][o][m] dense and active[n] in {0, 1}."""
    lib = _load()
    P = prob if isinstance(prob, Problem) else Problem(prob)
    S1 = np.empty((NDIR, 27, NDIR), np.float64)
    S0 = np.empty((NDIR, 27, NDIR), np.float64)
    act = np.empty(NDIR, np.int32)
    if lib.orc_two_step_stencil(ctypes.byref(P.s), int(k1), int(k2), _ptr(S1), _ptr(S0), _ptr(act)):
        raise ValueError("oracle: invalid problem or medium pair")
    return S1, S0, act


def fresnel(cos_i: float, n1: float, n2: float) -> float:
    return _load().orc_fresnel(float(cos_i), float(n1), float(n2))


def direction(d: int):
    out = np.zeros(3, np.int32)
    _load().orc_direction(int(d), _ptr(out))
    return tuple(int(v) for v in out)


def max_threads() -> int:
    lib = _load()
    lib.orc_max_threads.restype = ctypes.c_int
    return lib.orc_max_threads()
