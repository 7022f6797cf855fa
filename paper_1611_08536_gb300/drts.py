"""Thin ctypes binding of libdrts.so (C ABI in include/drts.h).

Argument marshalling only: every step of the time step runs in the library's
CUDA kernels.  Loading fails loudly when the library has not been built;
there is no CPU fallback.  PyTorch is used only to hand the library a CUDA
stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdrts.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE, EUNSUPPORTED = range(7)
OPEN, MIRROR, FRESNEL = 0, 1, 2
FP64, FP32, FP16_ROWSCALE = 0, 1, 2
FACE_NONE = -1
BATCHED_CUDA_CORES, BATCHED_TENSOR = 0, 1
FAULT_NONE, FAULT_SKIP_COPY, FAULT_SPIN_LIMIT, FAULT_SKIP_BARRIER = 0, 1, 2, 3
STEP_LAUNCH, STEP_PERSISTENT = 0, 1
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ESTATE",
           6: "EUNSUPPORTED"}


class DrtsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Medium(ctypes.Structure):
    _fields_ = [("mu_s", ctypes.c_double), ("mu_a", ctypes.c_double),
                ("g", ctypes.c_double), ("n", ctypes.c_double)]


# weights of the outgoing directions in the discrete HG kernel (drts.h)
HG_EQUAL, HG_QUADRATURE = 0, 1


class ProblemC(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("voxel_mm", ctypes.c_double),
        ("n_media", ctypes.c_int32),
        ("media", ctypes.POINTER(Medium)),
        ("medium_of_voxel", ctypes.c_void_p),
        ("n_outside", ctypes.c_double),
        ("boundary", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("n_rhs", ctypes.c_int32),
        ("det_face", ctypes.c_int32),
        ("det_nu", ctypes.c_int32), ("det_nv", ctypes.c_int32),
        ("max_steps", ctypes.c_int64),
        ("batched_kernel", ctypes.c_int32),
        ("interface", ctypes.c_int32),
        ("direction_weights", ctypes.c_int32),
    ]


class FccProblemC(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("spacing_mm", ctypes.c_double), ("n_media", ctypes.c_int32),
                ("media", ctypes.POINTER(Medium)), ("medium_of_site", ctypes.c_void_p)]


class TuneResult(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("rhs_tile", ctypes.c_int32),
                ("ms_per_step", ctypes.c_double), ("candidates", ctypes.c_int32),
                ("from_cache", ctypes.c_int32)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("max_resident", ctypes.c_int32),
                ("steps_per_tick", ctypes.c_int32), ("n_streams", ctypes.c_int32),
                ("policy", ctypes.c_int32), ("keep_state", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("n_rhs", ctypes.c_int32), ("n_patch", ctypes.c_int32),
                ("n_steps", ctypes.c_int64), ("footprint_bytes", ctypes.c_int64),
                ("queue_s", ctypes.c_double), ("latency_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("ticks", ctypes.c_int64), ("graph_launches", ctypes.c_int64),
                ("resident", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("used_bytes", ctypes.c_int64), ("budget_bytes", ctypes.c_int64),
                ("graph_updates", ctypes.c_int64), ("graph_instantiations", ctypes.c_int64),
                ("host_graph_s", ctypes.c_double), ("host_instantiate_s", ctypes.c_double),
                ("cancelled", ctypes.c_int64)]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [
        ("n_states", ctypes.c_int64), ("nnz", ctypes.c_int64),
        ("nnz_padded", ctypes.c_int64), ("n_slices", ctypes.c_int64),
        ("matrix_bytes", ctypes.c_int64), ("state_bytes", ctypes.c_int64),
        ("t", ctypes.c_int64),
        ("precision", ctypes.c_int32), ("n_rhs", ctypes.c_int32),
        ("n_patch", ctypes.c_int32), ("special_voxels_permille", ctypes.c_int32),
        ("nnz_stored", ctypes.c_int64),
    ]


SYMBOLS = ["drts_assemble", "drts_inject_source", "drts_step_n", "drts_read_detectors",
           "drts_read_state", "drts_write_state", "drts_run_host", "drts_export_rows",
           "drts_column_info", "drts_get_info", "drts_host_tables", "drts_two_step_tables", "drts_set_launch", "drts_destroy",
           "drts_last_error", "drts_state_sum_noalloc", "drts_set_fault", "drts_set_alloc_fault", "drts_set_allocator", "drts_autotune",
           "drts_set_step_mode", "drts_server_create", "drts_server_submit", "drts_server_tick",
           "drts_server_poll", "drts_server_result", "drts_server_result_state",
           "drts_server_cancel", "drts_server_release",
           "drts_server_get_stats", "drts_server_last_error", "drts_server_destroy",
           "drts_checkpoint_size", "drts_checkpoint_save", "drts_checkpoint_load",
           "drts_set_point_detectors", "drts_read_point_detectors", "drts_sensor_response",
           "drts_source_column", "drts_inject_source_substeps", "drts_substep_count",
           "drts_fcc_host_rows", "drts_fcc_assemble", "drts_fcc_set_source", "drts_fcc_step_n",
           "drts_fcc_read_state", "drts_fcc_read_rows", "drts_fcc_get_info", "drts_fcc_destroy"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libdrts.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libdrts.so not built ({path}); run "
                          "python -c 'import __graft_entry__ as g; g.build()'")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.drts_assemble.argtypes = [ctypes.POINTER(ProblemC), vp, ctypes.POINTER(vp)]
    lib.drts_inject_source.argtypes = [vp, i32, i32, vp, vp, i64, i32, vp]
    lib.drts_step_n.argtypes = [vp, i64]
    lib.drts_read_detectors.argtypes = [vp, i32, i64, i64, vp, vp]
    lib.drts_read_state.argtypes = [vp, i32, vp]
    lib.drts_write_state.argtypes = [vp, i32, vp]
    lib.drts_run_host.argtypes = [vp, i64, vp, vp]
    lib.drts_export_rows.argtypes = [vp, i64, i64, vp, vp, vp, i64]
    lib.drts_column_info.argtypes = [vp, vp, vp, vp]
    lib.drts_get_info.argtypes = [vp, ctypes.POINTER(Info)]
    lib.drts_host_tables.argtypes = [ctypes.POINTER(ProblemC), i32, vp, vp, vp, vp]
    lib.drts_two_step_tables.argtypes = [ctypes.POINTER(ProblemC), i32, i32, vp, vp, vp]
    lib.drts_fcc_host_rows.argtypes = [ctypes.POINTER(FccProblemC), i64, i64, vp, vp, vp, i64]
    lib.drts_fcc_assemble.argtypes = [ctypes.POINTER(FccProblemC), i32, vp, ctypes.POINTER(vp)]
    lib.drts_fcc_set_source.argtypes = [vp, i32, vp, vp, i64, i32, vp]
    lib.drts_fcc_step_n.argtypes = [vp, i64]
    lib.drts_fcc_read_state.argtypes = [vp, vp]
    lib.drts_fcc_read_rows.argtypes = [vp, i64, i64, vp, vp, vp, i64]
    lib.drts_fcc_get_info.argtypes = [vp, ctypes.POINTER(FccInfo)]
    lib.drts_fcc_destroy.argtypes = [vp]
    lib.drts_set_launch.argtypes = [vp, i32, i32, i32, i32]
    lib.drts_state_sum_noalloc.argtypes = [vp, i32, vp]
    lib.drts_set_fault.argtypes = [vp, i32, i64]
    lib.drts_autotune.argtypes = [vp, i32, ctypes.POINTER(TuneResult)]
    lib.drts_set_step_mode.argtypes = [vp, i32]
    lib.drts_checkpoint_size.argtypes = [vp, ctypes.POINTER(i64)]
    lib.drts_checkpoint_save.argtypes = [vp, vp, i64]
    lib.drts_checkpoint_load.argtypes = [vp, vp, i64]
    lib.drts_set_point_detectors.argtypes = [vp, i32, i64, vp, vp, vp]
    lib.drts_read_point_detectors.argtypes = [vp, i32, i64, i64, vp]
    lib.drts_sensor_response.argtypes = [vp, i32, i32, i64, i64, i32, vp, vp]
    lib.drts_source_column.argtypes = [vp, i64, ctypes.c_double, i32, vp, vp,
                                       ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]
    lib.drts_inject_source_substeps.argtypes = [vp, i32, i32, vp, vp, i32, i64, i32, vp]
    lib.drts_substep_count.argtypes = [vp, i64, ctypes.POINTER(i32)]
    lib.drts_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    lib.drts_server_submit.argtypes = [vp, ctypes.POINTER(ProblemC), i32, vp, vp, vp, i64, i32, vp,
                                       i64, ctypes.POINTER(i64)]
    lib.drts_server_tick.argtypes = [vp, ctypes.POINTER(i32)]
    lib.drts_server_poll.argtypes = [vp, i64, ctypes.POINTER(RequestInfo)]
    lib.drts_server_result.argtypes = [vp, i64, i32, vp, vp]
    lib.drts_server_result_state.argtypes = [vp, i64, i32, vp]
    lib.drts_server_cancel.argtypes = [vp, i64]
    lib.drts_set_alloc_fault.argtypes = [i64]
    lib.drts_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
    lib.drts_server_release.argtypes = [vp, i64]
    lib.drts_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    lib.drts_server_last_error.argtypes = [vp]
    lib.drts_server_last_error.restype = ctypes.c_char_p
    lib.drts_server_destroy.argtypes = [vp]
    lib.drts_server_destroy.restype = None
    lib.drts_destroy.argtypes = [vp]
    lib.drts_destroy.restype = None
    lib.drts_last_error.argtypes = [vp]
    lib.drts_last_error.restype = ctypes.c_char_p
    for name in SYMBOLS:
        getattr(lib, name)
    _lib = lib
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


# drts_alloc_fn / drts_free_fn
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_allocator_refs = None           # the installed callbacks, kept alive while installed


def use_torch_allocator():
    """Let PyTorch's caching allocator supply the device buffers of the
    contexts made from now on (drts_set_allocator): they count in
    torch.cuda.memory_allocated() and return to its cache on close."""
    import torch
    global _allocator_refs

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream) if stream else None)
        except Exception:          # out of memory: the library reports DRTS_ENOMEM
            return None

    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    refs = (ALLOC_FN(_alloc), FREE_FN(_free))
    st = load().drts_set_allocator(refs[0], refs[1], None)
    if st != OK:
        raise DrtsError(st, "drts_set_allocator")
    _allocator_refs = refs


def use_cuda_allocator():
    """Back to cudaMalloc / cudaFree for contexts made from now on.  Buffers
    already taken from another allocator still go back to it; keep its
    callbacks alive until those contexts are closed (this module keeps the
    last installed pair)."""
    load().drts_set_allocator(ALLOC_FN(), FREE_FN(), None)


def set_alloc_fault(n_ok):
    """After n_ok further device allocations of context buffers, the next one
    fails as out of memory (drts_set_alloc_fault); negative disarms."""
    load().drts_set_alloc_fault(int(n_ok))


def host_tables(prob, medium):
    """Host-built tables of one medium, computed without a device: the
    stencil W[n][o][m] (Eq. 18-21, before folding), the exit fractions
    exit_total[mask][n] and exit_det[mask][n] by face mask, and the FP16
    row scale per direction (drts_host_tables)."""
    lib = load()
    ps = problem_struct(prob, 0)
    W = np.empty((26, 27, 26), np.float64)
    ex = np.empty((27, 26), np.float64)
    ed = np.empty((27, 26), np.float64)
    sc = np.empty(26, np.float32)
    st = lib.drts_host_tables(ctypes.byref(ps), int(medium), _ptr(W), _ptr(ex), _ptr(ed), _ptr(sc))
    if st != OK:
        raise DrtsError(st, lib.drts_last_error(None).decode())
    return W, ex, ed, sc


def two_step_tables(prob, k1, k2):
    """Host-built two-step entries of a planar-interface problem, computed
    without a device (drts_two_step_tables): (cross[26], fold[26][27][26],
    edge[26][27][26]) for a state of medium k1 next to a z layer of k2."""
    lib = load()
    ps = problem_struct(prob, 0)
    cross = np.empty(26, np.uint8)
    fold = np.empty((26, 27, 26), np.float64)
    edge = np.empty((26, 27, 26), np.float64)
    st = lib.drts_two_step_tables(ctypes.byref(ps), int(k1), int(k2), _ptr(cross), _ptr(fold), _ptr(edge))
    if st != OK:
        raise DrtsError(st, lib.drts_last_error(None).decode())
    return cross, fold, edge


def fcc_host_rows(shape, spacing_mm, media, medium_of_site, row_begin=0, row_end=None, cap=None):
    """Rows of the close-packed partition's matrix A assembled on the host
    (drts_fcc_host_rows): (row_ptr, col, val) in CSR form."""
    lib = load()
    nx, ny, nz = shape
    n_states = nx * ny * nz // 2 * 12
    if row_end is None:
        row_end = n_states
    med = (Medium * len(media))(*[Medium(*m) for m in media])
    mos = np.ascontiguousarray(medium_of_site, dtype=np.uint8).ravel()
    p = FccProblemC(nx, ny, nz, float(spacing_mm), len(media), med, _ptr(mos))
    n = row_end - row_begin
    rp = np.zeros(max(n, 0) + 1, np.int64)
    if cap is None:
        cap = 700 * max(n, 0) + 16
    col = np.empty(cap, np.int32)
    val = np.empty(cap, np.float64)
    st = lib.drts_fcc_host_rows(ctypes.byref(p), int(row_begin), int(row_end), _ptr(rp), _ptr(col),
                                _ptr(val), int(cap))
    if st != OK:
        raise DrtsError(st, lib.drts_last_error(None).decode())
    nnz = int(rp[-1])
    return rp, col[:nnz].copy(), val[:nnz].copy()


class FccInfo(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int64), ("n_states", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("slots", ctypes.c_int64), ("n_offsets", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("t", ctypes.c_int64), ("matrix_bytes", ctypes.c_int64)]


class FccContext:
    """The Eq. 26 step on the close-packed partition, assembled and run on the
    device (drts_fcc_assemble ... drts_fcc_destroy); marshalling only."""

    def __init__(self, shape, spacing_mm, media, medium_of_site, precision=FP32, stream=None):
        self._lib = load()
        nx, ny, nz = shape
        self.shape = tuple(shape)
        self.n_states = nx * ny * nz // 2 * 12
        med = (Medium * len(media))(*[Medium(*m) for m in media])
        mos = np.ascontiguousarray(medium_of_site, dtype=np.uint8).ravel()
        p = FccProblemC(nx, ny, nz, float(spacing_mm), len(media), med, _ptr(mos))
        h = ctypes.c_void_p()
        st = self._lib.drts_fcc_assemble(ctypes.byref(p), int(precision), ctypes.c_void_p(stream), ctypes.byref(h))
        if st != OK:
            raise DrtsError(st, self._lib.drts_last_error(None).decode())
        self._h = h

    def _check(self, st):
        if st != OK:
            raise DrtsError(st, self._lib.drts_last_error(None).decode())

    def set_source(self, states, weights, profile, t0=0):
        st_ = np.ascontiguousarray(states, dtype=np.int64)
        w = np.ascontiguousarray(weights, dtype=np.float64)
        pr = np.ascontiguousarray(profile, dtype=np.float64)
        self._check(self._lib.drts_fcc_set_source(self._h, len(st_), _ptr(st_), _ptr(w), int(t0), len(pr),
                                                  _ptr(pr)))

    def step_n(self, n):
        self._check(self._lib.drts_fcc_step_n(self._h, int(n)))

    def read_state(self):
        out = np.empty(self.n_states, np.float64)
        self._check(self._lib.drts_fcc_read_state(self._h, _ptr(out)))
        return out

    def read_rows(self, row_begin=0, row_end=None, cap=None):
        if row_end is None:
            row_end = self.n_states
        n = row_end - row_begin
        rp = np.zeros(max(n, 0) + 1, np.int64)
        if cap is None:
            cap = 200 * max(n, 0) + 16
        col = np.empty(cap, np.int32)
        val = np.empty(cap, np.float64)
        self._check(self._lib.drts_fcc_read_rows(self._h, int(row_begin), int(row_end), _ptr(rp), _ptr(col),
                                                 _ptr(val), int(cap)))
        nnz = int(rp[-1])
        return rp, col[:nnz].copy(), val[:nnz].copy()

    def info(self):
        i = FccInfo()
        self._check(self._lib.drts_fcc_get_info(self._h, ctypes.byref(i)))
        return i

    def close(self):
        if getattr(self, "_h", None):
            self._lib.drts_fcc_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def problem_struct(prob, max_steps=0):
    """ctypes drts_problem for an ``inputs.Problem`` (keeps its buffers alive)."""
    media = (Medium * len(prob.media))(*[Medium(*m) for m in prob.media])
    mov = np.ascontiguousarray(prob.medium_of_voxel, dtype=np.uint8).ravel()
    nx, ny, nz = prob.shape
    s = ProblemC(nx, ny, nz, float(prob.voxel_mm), len(prob.media), media, _ptr(mov),
                 float(prob.n_outside), int(prob.boundary), int(prob.precision),
                 int(prob.n_rhs), int(prob.det_face), int(prob.det_nu),
                 int(prob.det_nv), int(max_steps), int(getattr(prob, "batched_kernel", 0)),
                 int(getattr(prob, "interface", 0)), int(getattr(prob, "direction_weights", 0)))
    s._keep = (media, mov)
    return s


class Context:
    """An assembled DRTS problem on the GPU (owns a drts_ctx)."""

    def __init__(self, prob, max_steps=0, stream=None):
        lib = load()
        self._lib = lib
        self.prob = prob
        self._ps = problem_struct(prob, max_steps)
        h = ctypes.c_void_p()
        st = lib.drts_assemble(ctypes.byref(self._ps), ctypes.c_void_p(stream or 0),
                               ctypes.byref(h))
        if st != OK:
            raise DrtsError(st, lib.drts_last_error(None).decode())
        self._h = h
        self.max_steps = max_steps
        self.n_states = prob.n_states

    def _check(self, st):
        if st != OK:
            raise DrtsError(st, self._lib.drts_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.drts_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- C ABI calls -------------------------------------------------------
    def inject_source(self, rhs, state_idx, weight, t0, profile):
        s = np.ascontiguousarray(state_idx, dtype=np.int64)
        w = np.ascontiguousarray(weight, dtype=np.float64)
        p = np.ascontiguousarray(profile, dtype=np.float64)
        self._check(self._lib.drts_inject_source(self._h, int(rhs), s.size, _ptr(s), _ptr(w),
                                                 int(t0), p.size, _ptr(p)))

    def set_source(self, rhs, src):
        self.inject_source(rhs, src.state, src.weight, src.t0, src.profile)

    def step_n(self, n):
        self._check(self._lib.drts_step_n(self._h, int(n)))

    def read_detectors(self, rhs=0, t_begin=0, t_end=None):
        info = self.info()
        if t_end is None:
            t_end = info.t
        out = np.zeros((max(t_end - t_begin, 0), max(info.n_patch, 1)), np.float64)
        led = np.zeros(4, np.float64)
        self._check(self._lib.drts_read_detectors(self._h, int(rhs), int(t_begin), int(t_end),
                                                  _ptr(out), _ptr(led)))
        return out[:, :info.n_patch], led

    def read_state(self, rhs=0):
        out = np.empty(self.n_states, np.float64)
        self._check(self._lib.drts_read_state(self._h, int(rhs), _ptr(out)))
        return out

    def write_state(self, x, rhs=0):
        x = np.ascontiguousarray(x, dtype=np.float64)
        if x.size != self.n_states:
            raise ValueError(f"state has {x.size} values, the problem {self.n_states}")
        self._check(self._lib.drts_write_state(self._h, int(rhs), _ptr(x)))

    def run_host(self, scale, det_out=None):
        scale = np.ascontiguousarray(scale, dtype=np.float64)
        n = scale.shape[0]
        self._check(self._lib.drts_run_host(self._h, n, _ptr(scale), _ptr(det_out)))
        return det_out

    def export_rows(self, row_begin, row_end, cap=None):
        n = row_end - row_begin
        rp = np.zeros(n + 1, np.int64)
        if cap is None:
            cap = 300 * n + 16
        col = np.empty(cap, np.int32)
        val = np.empty(cap, np.float64)
        self._check(self._lib.drts_export_rows(self._h, int(row_begin), int(row_end), _ptr(rp),
                                               _ptr(col), _ptr(val), int(cap)))
        nnz = int(rp[-1])
        return rp, col[:nnz].copy(), val[:nnz].copy()

    def column_info(self):
        ab, ex, ed = (np.empty(self.n_states, np.float64) for _ in range(3))
        self._check(self._lib.drts_column_info(self._h, _ptr(ab), _ptr(ex), _ptr(ed)))
        return ab, ex, ed

    def state_sum_noalloc(self, out_device_ptr, rhs=0):
        """Sum of x(t) into caller-owned device memory (one FP64 at
        ``out_device_ptr``), without any device allocation; asynchronous on
        the context stream."""
        self._check(self._lib.drts_state_sum_noalloc(self._h, int(rhs),
                                                     ctypes.c_void_p(int(out_device_ptr))))

    def autotune(self, trial_steps=3):
        """Time the launch candidates on the device and keep the fastest."""
        r = TuneResult()
        self._check(self._lib.drts_autotune(self._h, int(trial_steps), ctypes.byref(r)))
        return r.as_dict()

    def checkpoint(self) -> bytes:
        """t, states, ledger and detector history as bytes (A is not stored)."""
        n = ctypes.c_int64()
        self._check(self._lib.drts_checkpoint_size(self._h, ctypes.byref(n)))
        buf = np.empty(n.value, np.uint8)
        self._check(self._lib.drts_checkpoint_save(self._h, _ptr(buf), n.value))
        return buf.tobytes()

    def set_point_detectors(self, n_det, det, state_idx, weight):
        """Sparse detector rows F of Eq. 27: detector det[e] reads
        weight[e] * x_t[state_idx[e]], summed per detector every step."""
        d = np.ascontiguousarray(det, dtype=np.int32)
        st = np.ascontiguousarray(state_idx, dtype=np.int64)
        w = np.ascontiguousarray(weight, dtype=np.float64)
        if not (d.size == st.size == w.size):
            raise ValueError("det, state_idx and weight differ in length")
        self._check(self._lib.drts_set_point_detectors(self._h, int(n_det), d.size, _ptr(d),
                                                       _ptr(st), _ptr(w)))
        self._n_pdet = int(n_det)

    def read_point_detectors(self, rhs=0, t_begin=0, t_end=None):
        if t_end is None:
            t_end = self.info().t
        out = np.zeros((max(t_end - t_begin, 0), max(getattr(self, "_n_pdet", 0), 1)), np.float64)
        self._check(self._lib.drts_read_point_detectors(self._h, int(rhs), int(t_begin), int(t_end),
                                                        _ptr(out)))
        return out[:, :getattr(self, "_n_pdet", 0)]

    def sensor_response(self, w, h, rhs=0, which=0, t_begin=0, t_end=None, n_det=None):
        """Eq. 27 sensor output M[t][d] = sum_{|t-k| <= w} h[t-k+w] D[k][d] of the
        face (which=SENSOR_FACE) or point (SENSOR_POINT) detector history."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        if h.size != 2 * w + 1:
            raise ValueError("h must have 2w+1 taps")
        if t_end is None:
            t_end = self.info().t
        if n_det is None:
            n_det = self.info().n_patch if which == SENSOR_FACE else getattr(self, "_n_pdet", 0)
        out = np.zeros((max(t_end - t_begin, 0), max(n_det, 1)), np.float64)
        self._check(self._lib.drts_sensor_response(self._h, int(rhs), int(which), int(t_begin),
                                                   int(t_end), int(w), _ptr(h), _ptr(out)))
        return out[:, :n_det]

    def source_column(self, state_idx, frac, cap=4096):
        """(states, values, exit_mass) of a unit population emitted from
        state_idx that travels the fraction frac of a step (Section 4.1)."""
        st = np.empty(cap, np.int64)
        val = np.empty(cap, np.float64)
        cnt = ctypes.c_int32()
        ex = ctypes.c_double()
        self._check(self._lib.drts_source_column(self._h, int(state_idx), float(frac), int(cap),
                                                 _ptr(st), _ptr(val), ctypes.byref(cnt),
                                                 ctypes.byref(ex)))
        return st[:cnt.value].copy(), val[:cnt.value].copy(), ex.value

    def substep_count(self, state_idx):
        """Sub-intervals of length dr/c in one step of state_idx's medium."""
        n = ctypes.c_int32()
        self._check(self._lib.drts_substep_count(self._h, int(state_idx), ctypes.byref(n)))
        return n.value

    def inject_source_substeps(self, rhs, state_idx, weight, t0, profile):
        """Sub-step source of rhs: profile[t - t0][j] is emitted in sub-interval
        j of step t; n_sub is the profile's second extent."""
        s = np.ascontiguousarray(state_idx, dtype=np.int64)
        w = np.ascontiguousarray(weight, dtype=np.float64)
        p = np.ascontiguousarray(profile, dtype=np.float64)
        if p.ndim != 2:
            raise ValueError("profile must be [n_t][n_sub]")
        self._check(self._lib.drts_inject_source_substeps(self._h, int(rhs), s.size, _ptr(s), _ptr(w),
                                                          p.shape[1], int(t0), p.shape[0], _ptr(p)))

    def restore(self, data: bytes):
        buf = np.frombuffer(data, np.uint8).copy()
        self._check(self._lib.drts_checkpoint_load(self._h, _ptr(buf), buf.size))

    def set_step_mode(self, mode):
        """STEP_LAUNCH (one launch per step) or STEP_PERSISTENT (one
        cooperative launch for all steps of a drts_step_n call)."""
        self._check(self._lib.drts_set_step_mode(self._h, int(mode)))

    def set_fault(self, kind, arg=0):
        """Host-side fault injection (FAULT_NONE / FAULT_SKIP_COPY / FAULT_SPIN_LIMIT)."""
        self._check(self._lib.drts_set_fault(self._h, int(kind), int(arg)))

    def info(self):
        i = Info()
        self._check(self._lib.drts_get_info(self._h, ctypes.byref(i)))
        return i

    def set_launch(self, blocks_per_sm=0, threads=0, rhs_tile=0, variant=-1):
        self._check(self._lib.drts_set_launch(self._h, int(blocks_per_sm), int(threads),
                                              int(rhs_tile), int(variant)))


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = 0, 1, 2, 3, 4
SENSOR_FACE, SENSOR_POINT = 0, 1
SERVE_FIFO, SERVE_SHORTEST_FIRST = 0, 1


class Server:
    """Continuous-batching server of DRTS simulations (drts_server_*)."""

    def __init__(self, mem_budget_bytes=0, max_resident=16, steps_per_tick=10, n_streams=4,
                 policy=0, keep_state=False):
        """policy: SERVE_FIFO (arrival order) or SERVE_SHORTEST_FIRST;
        keep_state: keep every finished request's final states for
        ``result_state``."""
        self._lib = load()
        cfg = ServerConfig(int(mem_budget_bytes), int(max_resident), int(steps_per_tick),
                           int(n_streams), int(policy), int(bool(keep_state)), 0)
        h = ctypes.c_void_p()
        st = self._lib.drts_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise DrtsError(st, "drts_server_create failed")
        self._h = h

    def _check(self, st):
        if st != OK:
            raise DrtsError(st, self._lib.drts_server_last_error(self._h).decode())

    def submit(self, prob, sources, n_steps):
        """``sources``: list of inputs.Source, one per right-hand side (all
        sharing the first source's time profile)."""
        ps = problem_struct(prob, n_steps)
        rhs = np.concatenate([np.full(s.state.size, r, np.int32) for r, s in enumerate(sources)])
        st_ = np.concatenate([s.state for s in sources]).astype(np.int64)
        w = np.concatenate([s.weight for s in sources]).astype(np.float64)
        prof = np.ascontiguousarray(sources[0].profile, dtype=np.float64)
        rid = ctypes.c_int64()
        self._check(self._lib.drts_server_submit(self._h, ctypes.byref(ps), rhs.size, _ptr(rhs),
                                                 _ptr(st_), _ptr(w), int(sources[0].t0), prof.size,
                                                 _ptr(prof), int(n_steps), ctypes.byref(rid)))
        return rid.value

    def tick(self):
        n = ctypes.c_int32()
        self._check(self._lib.drts_server_tick(self._h, ctypes.byref(n)))
        return n.value

    def poll(self, rid):
        info = RequestInfo()
        self._check(self._lib.drts_server_poll(self._h, int(rid), ctypes.byref(info)))
        return info

    def result(self, rid, rhs=0):
        info = self.poll(rid)
        det = np.zeros((info.n_steps, max(info.n_patch, 1)), np.float64)
        led = np.zeros(4, np.float64)
        self._check(self._lib.drts_server_result(self._h, int(rid), int(rhs), _ptr(det), _ptr(led)))
        return det[:, :info.n_patch], led

    def result_state(self, rid, rhs=0, n_states=None):
        """Final state x(n_steps) of right-hand side rhs (canonical order);
        the server must keep states (``keep_state=True``)."""
        if n_states is None:
            raise ValueError("n_states is required (the problem's 26 * voxels)")
        out = np.empty(int(n_states), np.float64)
        self._check(self._lib.drts_server_result_state(self._h, int(rid), int(rhs), _ptr(out)))
        return out

    def cancel(self, rid):
        """Withdraw a queued or running request (drts_server_cancel)."""
        self._check(self._lib.drts_server_cancel(self._h, int(rid)))

    def release(self, rid):
        self._check(self._lib.drts_server_release(self._h, int(rid)))

    def stats(self):
        st = ServerStats()
        self._check(self._lib.drts_server_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            self._lib.drts_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def assemble(prob, max_steps=0, stream=None) -> Context:
    return Context(prob, max_steps=max_steps, stream=stream)


__all__ = ["Context", "assemble", "load", "DrtsError", "SYMBOLS", "_inputs"]
