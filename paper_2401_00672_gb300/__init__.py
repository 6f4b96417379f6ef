"""GB300 OBK-RCM: Python binding of the C ABI in ``include/obk.h``.

Argument marshalling only: every step of the method (extension, RCM, grouping,
sweeps, residual checks, refinement, request loop) runs in ``libobk.so``'s CUDA
kernels.  Arrays may be numpy arrays (host memory) or CUDA torch tensors (device
memory of the current device); PyTorch is used only for device memory and
streams.  There is no CPU fallback: importing this package without the built
library raises ``ImportError``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libobk.so")

OBK_OK, OBK_NOT_CONVERGED, OBK_PENDING = 0, 1, 2
OBK_ERR_INVALID, OBK_ERR_NOMEM, OBK_ERR_BUDGET = -1, -2, -3
OBK_ERR_TIMEOUT, OBK_ERR_CUDA, OBK_ERR_CANCELLED, OBK_ERR_NOT_FOUND = -4, -5, -6, -7

EXPORTS = [
    "obk_create", "obk_create_on_stream", "obk_solve", "obk_solve_ex", "obk_get_dims", "obk_get_perm",
    "obk_get_groups", "obk_get_row_norms", "obk_get_info", "obk_destroy", "obk_server_create",
    "obk_submit", "obk_poll", "obk_cancel", "obk_server_destroy", "obk_last_error", "obk_version",
    "obk_kernel_launches", "obk_residual", "obk_residual_noalloc", "obk_autotune", "obk_solve_batch",
    "obk_batch_max_n", "obk_get_setup_profile", "obk_grouping_stats", "obk_solve_blocks",
    "obk_request_footprint", "obk_measure_peaks", "obk_select_threshold",
]


class ObkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class _Csr(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("nnz", ctypes.c_int64), ("device_ptrs", ctypes.c_int32)]


class Opts(ctypes.Structure):
    """obk_opts (see include/obk.h); zero fields take the library defaults."""
    _fields_ = [("precision", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("inner_sweeps", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("stagnation", ctypes.c_double), ("timeout_spins", ctypes.c_int64),
                ("rows_per_warp", ctypes.c_int32), ("pinv_iters", ctypes.c_int32),
                ("sync_mode", ctypes.c_int32), ("staging", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _GStats(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("nonzero_entries", ctypes.c_int64), ("abs_cos_sum", ctypes.c_uint64),
                ("zn", ctypes.c_double), ("nn", ctypes.c_double), ("groups", ctypes.c_int64),
                ("min_group_rows", ctypes.c_int64), ("max_group_rows", ctypes.c_int64),
                ("conflicts", ctypes.c_int64), ("color_rounds", ctypes.c_int64), ("reserved", ctypes.c_int64 * 2)]


class BlockOpts(ctypes.Structure):
    """obk_block_opts (see include/obk.h)."""
    _fields_ = [("k", ctypes.c_int32), ("inner_max", ctypes.c_int32), ("thr", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("n_pairs", ctypes.c_int32), ("n_nclass", ctypes.c_int32),
                ("cgls_steps", ctypes.c_int64), ("reserved", ctypes.c_int64 * 2)]


class _Tune(ctypes.Structure):
    _fields_ = [("rows_per_warp", ctypes.c_int32), ("block_threads", ctypes.c_int32), ("staging", ctypes.c_int32),
                ("sync_mode", ctypes.c_int32), ("n_candidates", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("sweep_ms", ctypes.c_double), ("candidate_ms", ctypes.c_double * 16)]


class _Info(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("rel_res", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("groups", ctypes.c_int64),
                ("bandwidth_before", ctypes.c_int64), ("bandwidth_after", ctypes.c_int64),
                ("outer_iters", ctypes.c_int64), ("sweep_ms", ctypes.c_double),
                ("n_conflicts", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]


@dataclasses.dataclass
class Info:
    sweeps: int
    rel_res: float
    setup_ms: float
    solve_ms: float
    groups: int
    bandwidth_before: int
    bandwidth_after: int
    outer_iters: int
    sweep_ms: float
    n_conflicts: int
    status: int


def _info(ci: _Info) -> Info:
    return Info(*(getattr(ci, f[0]) for f in _Info._fields_ if f[0] != "reserved"))


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libobk.so is not built ({LIB_PATH}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "obk_create": ([vp, i64, i64, dbl, vp], ctypes.c_int),
        "obk_create_on_stream": ([vp, i64, i64, dbl, vp, vp], ctypes.c_int),
        "obk_solve": ([vp, vp, vp, dbl, i64, vp, vp], ctypes.c_int),
        "obk_solve_ex": ([vp, vp, vp, vp, dbl, i64, vp, vp], ctypes.c_int),
        "obk_get_dims": ([vp, vp, vp, vp], ctypes.c_int),
        "obk_get_perm": ([vp, vp], ctypes.c_int),
        "obk_get_groups": ([vp, vp], ctypes.c_int),
        "obk_get_row_norms": ([vp, vp], ctypes.c_int),
        "obk_get_info": ([vp, vp], ctypes.c_int),
        "obk_destroy": ([vp], None),
        "obk_server_create": ([ctypes.c_size_t, i32, vp], ctypes.c_int),
        "obk_submit": ([vp, vp, i64, i64, dbl, vp, vp, dbl, i64, vp, vp], ctypes.c_int),
        "obk_poll": ([vp, ctypes.c_uint64, vp, vp], ctypes.c_int),
        "obk_cancel": ([vp, ctypes.c_uint64], ctypes.c_int),
        "obk_server_destroy": ([vp], None),
        "obk_last_error": ([], ctypes.c_char_p),
        "obk_version": ([], ctypes.c_char_p),
        "obk_kernel_launches": ([], ctypes.c_int64),
        "obk_residual": ([vp, i64, i64, vp, vp, vp], ctypes.c_int),
        "obk_residual_noalloc": ([vp, vp, vp, i64, i64, vp, vp, vp, vp], ctypes.c_int),
        "obk_autotune": ([vp, i32, vp], ctypes.c_int),
        "obk_solve_batch": ([vp, i32, vp, vp, vp, dbl, i64, vp, vp, vp], ctypes.c_int),
        "obk_batch_max_n": ([], ctypes.c_int64),
        "obk_get_setup_profile": ([vp, vp, i32], ctypes.c_int32),
        "obk_grouping_stats": ([vp, vp], ctypes.c_int32),
        "obk_solve_blocks": ([vp, vp, vp, vp, dbl, i64, vp, vp], ctypes.c_int32),
        "obk_request_footprint": ([i64, i64, i64], ctypes.c_size_t),
        "obk_measure_peaks": ([vp], ctypes.c_int),
        "obk_select_threshold": ([vp, i64, i64, vp, vp, i32, i32, dbl, vp, vp, vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


class _Peaks(ctypes.Structure):
    _fields_ = [("fp64_fma_tflops", ctypes.c_double), ("fp32_fma_tflops", ctypes.c_double),
                ("l2_gather_g_per_s", ctypes.c_double), ("l2_read_gbs", ctypes.c_double),
                ("int64_mad_tops", ctypes.c_double), ("int32_mad_tops", ctypes.c_double)]


def measure_peaks() -> dict:
    """obk_measure_peaks: FP64/FP32 multiply-add rates, L2 gather and read rates."""
    p = _Peaks()
    _check(lib.obk_measure_peaks(ctypes.byref(p)), "obk_measure_peaks")
    return {f[0]: getattr(p, f[0]) for f in _Peaks._fields_}


class _ThrProbe(ctypes.Structure):
    _fields_ = [("thr", ctypes.c_double), ("groups", ctypes.c_int64), ("conflicts", ctypes.c_int64),
                ("probe_sweeps", ctypes.c_int64), ("setup_ms", ctypes.c_double), ("probe_ms", ctypes.c_double),
                ("rel_res", ctypes.c_double), ("rate", ctypes.c_double), ("predicted_ms", ctypes.c_double)]


def select_threshold(row_ptr, col_idx, val, m, n, f, candidates=(0.02, 0.05, 0.1, 0.2, 0.3), probe_sweeps=6,
                     tol=1e-8, keep_handle=True):
    """obk_select_threshold: the candidate thr with the smallest predicted time
    to tol from a short FP64 probe solve at each.  Returns (thr, Handle or None,
    list of per-candidate dicts)."""
    p_rp, dev, k1 = _ptr(row_ptr, np.int64)
    p_ci, _, k2 = _ptr(col_idx, np.int32)
    p_v, _, k3 = _ptr(val, np.float64)
    nnz = int(k1[-1]) if not dev else int(k1[-1].item())
    csr = _Csr(p_rp, p_ci, p_v, nnz, 1 if dev else 0)
    pf, _, kf = _ptr(f, np.float64)
    cand = np.ascontiguousarray(candidates, dtype=np.float64)
    probes = (_ThrProbe * len(cand))()
    thr = ctypes.c_double()
    hv = ctypes.c_void_p()
    _check(lib.obk_select_threshold(ctypes.byref(csr), int(m), int(n), pf, cand.ctypes.data_as(ctypes.c_void_p),
                                    len(cand), int(probe_sweeps), float(tol), ctypes.byref(thr),
                                    ctypes.byref(hv) if keep_handle else None, probes), "obk_select_threshold")
    h = None
    if keep_handle:
        h = Handle.__new__(Handle)
        h._h = hv
        h._csr = csr
        h.m, h.n = m, n
        N, nz, G = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        lib.obk_get_dims(hv, ctypes.byref(N), ctypes.byref(nz), ctypes.byref(G))
        h.N, h.nnz, h.G = N.value, nz.value, G.value
    rows = [{k: getattr(pr, k) for k, _ in _ThrProbe._fields_} for pr in probes]
    return thr.value, h, rows


def request_footprint(m: int, n: int, nnz: int) -> int:
    """obk_request_footprint: HBM bytes the request loop reserves for such a request."""
    return int(lib.obk_request_footprint(int(m), int(n), int(nnz)))


def kernel_launches() -> int:
    """CUDA kernels launched by libobk.so in this process so far."""
    return int(lib.obk_kernel_launches())


def last_error() -> str:
    return lib.obk_last_error().decode()


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise ObkError(rc, f"{what}: {last_error()}")
    return rc


def _ptr(a, dtype):
    """(pointer, is_device, keepalive) for a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, False, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        import torch

        want = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return ctypes.c_void_p(a.data_ptr()), bool(a.is_cuda), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), False, arr


class Handle:
    """One system A (m x n) prepared on the GPU: obk_create ... obk_destroy."""

    def __init__(self, row_ptr, col_idx, val, m: int, n: int, thr: float = 0.1, stream=None):
        p_rp, d1, k1 = _ptr(row_ptr, np.int64)
        p_ci, d2, k2 = _ptr(col_idx, np.int32)
        p_v, d3, k3 = _ptr(val, np.float64)
        if not (d1 == d2 == d3):
            raise TypeError("row_ptr, col_idx and val must all be host or all be device arrays")
        nnz = int(k1[-1]) if not d1 else int(k1[-1].item())
        self._csr = _Csr(p_rp, p_ci, p_v, nnz, 1 if d1 else 0)
        self._h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream else None
        _check(lib.obk_create_on_stream(ctypes.byref(self._csr), m, n, float(thr), st, ctypes.byref(self._h)),
               "obk_create")
        self.m, self.n = m, n
        N, nz, G = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        lib.obk_get_dims(self._h, ctypes.byref(N), ctypes.byref(nz), ctypes.byref(G))
        self.N, self.nnz, self.G = N.value, nz.value, G.value

    def solve(self, f, x0=None, tol: float = 1e-8, maxit: int = 1000, out=None, opts: Opts | None = None):
        """Returns (status, x, Info); x is numpy unless `out` (a CUDA tensor) is given."""
        pf, _, kf = _ptr(f, np.float64)
        px, _, kx = _ptr(x0, np.float64)
        if out is None:
            out = np.empty(self.n, np.float64)
        po, _, ko = _ptr(out, np.float64)
        info = _Info()
        rc = lib.obk_solve_ex(self._h, ctypes.byref(opts) if opts is not None else None, pf, px, float(tol),
                              int(maxit), po, ctypes.byref(info))
        _check(rc, "obk_solve")
        return rc, ko, _info(info)

    SETUP_STAGES = ("upload_validate_extend", "bandwidth_in", "rcm_graph", "rcm_ranks", "rcm_search",
                    "rcm_cuthill_mckee", "permute", "norms_transpose",
                    "pair_cosines", "grouping", "group_rows", "mirror_segments", "bookkeeping")

    def solve_blocks(self, f, x0=None, k: int = 8, thr: float = 0.0, tol: float = 1e-8, maxit: int = 1000,
                     inner_max: int = 0, inner_tol: float = 0.0, out=None):
        """obk_solve_blocks (Algorithm 4 as printed).  Returns (status, x, Info, BlockOpts)."""
        pf, _, kf = _ptr(f, np.float64)
        px, _, kx = _ptr(x0, np.float64)
        if out is None:
            out = np.empty(self.n, np.float64)
        po, _, ko = _ptr(out, np.float64)
        bo = BlockOpts(k=k, inner_max=inner_max, thr=thr, inner_tol=inner_tol)
        info = _Info()
        rc = lib.obk_solve_blocks(self._h, ctypes.byref(bo), pf, px, float(tol), int(maxit), po, ctypes.byref(info))
        _check(rc, "obk_solve_blocks")
        return rc, ko, _info(info), bo

    def grouping_stats(self) -> dict:
        """obk_grouping_stats: Definitions 1-2 (zn, nn) of the row cosine table, group sizes,
        conflict count and grouping rounds."""
        g = _GStats()
        _check(lib.obk_grouping_stats(self._h, ctypes.byref(g)), "obk_grouping_stats")
        return {k: getattr(g, k) for k, _ in _GStats._fields_ if k != "reserved"}

    def setup_profile(self) -> dict:
        """obk_get_setup_profile: device milliseconds per obk_create stage."""
        ms = (ctypes.c_double * 16)()
        n = lib.obk_get_setup_profile(self._h, ms, 16)
        return {name: round(ms[i], 4) for i, name in enumerate(self.SETUP_STAGES[:n])}

    TUNE_CANDIDATES = ((32, 1024, "counters", "global"), (32, 1024, "counters", "shared"),
                       (32, 512, "counters", "global"), (32, 512, "counters", "shared"),
                       (32, 1024, "barriers", "global"), (32, 512, "barriers", "global"),
                       (16, 1024, "barriers", "global"), (16, 512, "barriers", "global"),
                       (8, 1024, "barriers", "global"), (8, 512, "barriers", "global"),
                       (4, 1024, "barriers", "global"), (4, 512, "barriers", "global"),
                       (2, 1024, "barriers", "global"), (2, 512, "barriers", "global"))

    def autotune(self, precision: int = 0) -> dict:
        """obk_autotune: time the (rows per warp, threads per block, ordering,
        x/y placement) settings and keep the fastest.  candidate_ms maps each
        timed setting to its sweep time (0 = skipped)."""
        t = _Tune()
        _check(lib.obk_autotune(self._h, int(precision), ctypes.byref(t)), "obk_autotune")
        return {"rows_per_warp": t.rows_per_warp, "block_threads": t.block_threads,
                "sync": "counters" if t.sync_mode == 2 else "barriers",
                "staging": "shared" if t.staging == 1 else "global", "sweep_ms": t.sweep_ms,
                "candidate_ms": dict(zip(self.TUNE_CANDIDATES, list(t.candidate_ms)[: t.n_candidates]))}

    def _get(self, fn, dtype):
        a = np.empty(self.N, dtype)
        _check(fn(self._h, a.ctypes.data_as(ctypes.c_void_p)), fn.__name__)
        return a

    def perm(self) -> np.ndarray:
        return self._get(lib.obk_get_perm, np.int32)

    def groups(self) -> np.ndarray:
        return self._get(lib.obk_get_groups, np.int32)

    def row_norms(self) -> np.ndarray:
        return self._get(lib.obk_get_row_norms, np.float64)

    def info(self) -> Info:
        i = _Info()
        _check(lib.obk_get_info(self._h, ctypes.byref(i)), "obk_get_info")
        return _info(i)

    def close(self):
        if self._h:
            lib.obk_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def residual(row_ptr, col_idx, val, m, n, f, x) -> float:
    """obk_residual: ||f - A x|| / ||f|| in FP64 (deterministic tile reduction)."""
    p_rp, dev, k1 = _ptr(row_ptr, np.int64)
    p_ci, _, k2 = _ptr(col_idx, np.int32)
    p_v, _, k3 = _ptr(val, np.float64)
    nnz = int(k1[-1]) if not dev else int(k1[-1].item())
    csr = _Csr(p_rp, p_ci, p_v, nnz, 1 if dev else 0)
    pf, _, kf = _ptr(f, np.float64)
    px, _, kx = _ptr(x, np.float64)
    out = ctypes.c_double()
    _check(lib.obk_residual(ctypes.byref(csr), m, n, pf, px, ctypes.byref(out)), "obk_residual")
    return out.value


def residual_noalloc(row_ptr, col_idx, val, m, n, f, x, out, stream=None) -> int:
    """obk_residual_noalloc: all arguments are CUDA tensors of the current
    device (out: one float64); queued on `stream` (raw cudaStream_t handle,
    None = default stream).  An empty col_idx / val (a matrix without entries)
    is passed as a one-element device buffer: the C entry point rejects NULL."""
    import torch

    cur = torch.cuda.current_device()
    ptrs, keep = [], []
    for a, dt in ((row_ptr, np.int64), (col_idx, np.int32), (val, np.float64), (f, np.float64),
                  (x, np.float64), (out, np.float64)):
        if hasattr(a, "is_cuda") and a.is_cuda and a.numel() == 0:
            a = torch.zeros(1, dtype=a.dtype, device=a.device)
            keep.append(a)
        p, dev, _ = _ptr(a, dt)
        if not dev:
            raise TypeError("obk_residual_noalloc takes device arrays only")
        if a.device.index != cur:
            raise TypeError(f"obk_residual_noalloc: array on {a.device}, current device is cuda:{cur}")
        ptrs.append(p)
    return _check(lib.obk_residual_noalloc(ptrs[0], ptrs[1], ptrs[2], int(m), int(n), ptrs[3], ptrs[4], ptrs[5],
                                           ctypes.c_void_p(stream) if stream else None), "obk_residual_noalloc")


def solve_batch(handles, fs, outs, x0s=None, tol=1e-8, maxit=1000, opts=None):
    """obk_solve_batch: one launch for several prepared systems (device tensors).
    Returns (statuses, infos)."""
    n = len(handles)
    H = (ctypes.c_void_p * n)(*[h._h.value for h in handles])
    F = (ctypes.c_void_p * n)(*[_ptr(a, np.float64)[0].value for a in fs])
    X = (ctypes.c_void_p * n)(*[_ptr(a, np.float64)[0].value for a in outs])
    X0 = None
    if x0s is not None:
        X0 = (ctypes.c_void_p * n)(*[(_ptr(a, np.float64)[0].value if a is not None else None) for a in x0s])
    infos = (_Info * n)()
    sts = (ctypes.c_int * n)()
    _check(lib.obk_solve_batch(H, n, ctypes.byref(opts) if opts is not None else None, F, X0, float(tol), int(maxit),
                               X, infos, sts), "obk_solve_batch")
    return list(sts), [_info(i) for i in infos]


def solve(row_ptr, col_idx, val, m, n, f, x0=None, thr=0.1, tol=1e-8, maxit=1000, opts=None):
    """One-shot obk_create + obk_solve + obk_destroy; returns (status, x, Info)."""
    with Handle(row_ptr, col_idx, val, m, n, thr) as h:
        return h.solve(f, x0, tol, maxit, opts=opts)


class Server:
    """Request loop (obk_server_*): submit systems, poll for results."""

    def __init__(self, hbm_budget_bytes: int = 0, max_streams: int = 0):
        self._s = ctypes.c_void_p()
        _check(lib.obk_server_create(int(hbm_budget_bytes), int(max_streams), ctypes.byref(self._s)),
               "obk_server_create")

    def submit(self, row_ptr, col_idx, val, m, n, f, x0=None, thr=0.1, tol=1e-8, maxit=1000,
               opts: Opts | None = None) -> int:
        p_rp, dev, k1 = _ptr(row_ptr, np.int64)
        p_ci, _, k2 = _ptr(col_idx, np.int32)
        p_v, _, k3 = _ptr(val, np.float64)
        nnz = int(k1[-1]) if not dev else int(k1[-1].item())
        csr = _Csr(p_rp, p_ci, p_v, nnz, 1 if dev else 0)
        pf, _, kf = _ptr(f, np.float64)
        px, _, kx = _ptr(x0, np.float64)
        t = ctypes.c_uint64()
        _check(lib.obk_submit(self._s, ctypes.byref(csr), m, n, float(thr), pf, px, float(tol), int(maxit),
                              ctypes.byref(opts) if opts is not None else None, ctypes.byref(t)), "obk_submit")
        return t.value

    def poll(self, ticket: int, n: int):
        """(status, x or None, Info or None); status OBK_PENDING while running."""
        x = np.empty(n, np.float64)
        info = _Info()
        rc = lib.obk_poll(self._s, ctypes.c_uint64(ticket), x.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info))
        if rc == OBK_PENDING:
            return rc, None, None
        return rc, x, _info(info)

    def cancel(self, ticket: int) -> int:
        return lib.obk_cancel(self._s, ctypes.c_uint64(ticket))

    def close(self):
        if self._s:
            lib.obk_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
