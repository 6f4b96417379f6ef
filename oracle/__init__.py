"""CPU oracle for OBK-RCM (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never touches it, and it shares no code with that path.

``obk_oracle.c`` is plain single-threaded C compiled with
``-ffp-contract=off``; this module compiles it on first use (or through
``build()``) and wraps it with ctypes over numpy arrays.

Every function here follows a step of the paper (Liang & Li, OBK-RCM,
arXiv 2401.00672); the C file's header maps each to its section/equation.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "obk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, NOT_CONVERGED, INVALID, NOMEM = 0, 1, -1, -2


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no FP contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Info(ctypes.Structure):
    _fields_ = [
        ("sweeps", ctypes.c_int64),
        ("rel_res", ctypes.c_double),
        ("groups", ctypes.c_int64),
        ("bandwidth_before", ctypes.c_int64),
        ("bandwidth_after", ctypes.c_int64),
        ("n_conflicts", ctypes.c_int64),
        ("outer_iters", ctypes.c_int64),
        ("status", ctypes.c_int64),
    ]


class _Opts(ctypes.Structure):
    _fields_ = [
        ("check_every", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("inner_sweeps", ctypes.c_int32),
        ("max_outer", ctypes.c_int32),
        ("stagnation", ctypes.c_double),
        ("pinv_iters", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.orc_residual.restype = ctypes.c_double
            _lib.orc_bandwidth.restype = ctypes.c_int64
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(rp, ci, v):
    return (np.ascontiguousarray(rp, dtype=np.int64), np.ascontiguousarray(ci, dtype=np.int32),
            np.ascontiguousarray(v, dtype=np.float64))


@dataclasses.dataclass
class Info:
    sweeps: int
    rel_res: float
    groups: int
    bandwidth_before: int
    bandwidth_after: int
    n_conflicts: int
    outer_iters: int
    status: int


def _info(ci: _Info) -> Info:
    return Info(*(getattr(ci, f[0]) for f in _Info._fields_))


def validate(m, n, rp, ci, v) -> int:
    rp, ci, v = _csr(rp, ci, v)
    return _load().orc_validate(ctypes.c_int64(m), ctypes.c_int64(n), _p(rp), _p(ci), _p(v),
                                ctypes.c_int64(int(rp[-1])))


def rcm(N, rp, ci) -> np.ndarray:
    """perm[k] = old index at new position k (Reverse Cuthill-McKee, Section 3.2)."""
    rp, ci, _ = _csr(rp, ci, np.zeros(0))
    perm = np.empty(N, dtype=np.int32)
    rc = _load().orc_rcm(ctypes.c_int64(N), _p(rp), _p(ci), _p(perm))
    if rc:
        raise MemoryError("oracle rcm failed")
    return perm


def bandwidth(N, rp, ci) -> int:
    rp, ci, _ = _csr(rp, ci, np.zeros(0))
    return int(_load().orc_bandwidth(ctypes.c_int64(N), _p(rp), _p(ci)))


def permute(N, rp, ci, v, perm):
    """A~ = P A P^T (Eq. 3.1) with columns re-sorted in each row."""
    rp, ci, v = _csr(rp, ci, v)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    nnz = int(rp[-1])
    rpo = np.empty(N + 1, np.int64)
    cio = np.empty(max(nnz, 1), np.int32)
    vo = np.empty(max(nnz, 1), np.float64)
    rc = _load().orc_permute(ctypes.c_int64(N), _p(rp), _p(ci), _p(v), _p(perm), _p(rpo),
                             _p(cio), _p(vo))
    if rc:
        raise MemoryError("oracle permute failed")
    return rpo, cio[:nnz], vo[:nnz]


def row_norms(N, rp, v) -> np.ndarray:
    rp, _, v = _csr(rp, np.zeros(0), v)
    out = np.empty(N, np.float64)
    _load().orc_row_norms(ctypes.c_int64(N), _p(rp), _p(v), _p(out))
    return out


def group_build(N, rp, ci, v, nsq, thr):
    """Greedy first-fit groups under |cos| >= thr conflicts (Section 3.3, k = m).
    Returns (group_of int32[N] with -1 for zero rows, G, n_conflicts)."""
    rp, ci, v = _csr(rp, ci, v)
    nsq = np.ascontiguousarray(nsq, np.float64)
    gof = np.empty(N, np.int32)
    G = ctypes.c_int64(0)
    nc = ctypes.c_int64(0)
    rc = _load().orc_group_build(ctypes.c_int64(N), _p(rp), _p(ci), _p(v), _p(nsq),
                                 ctypes.c_double(thr), _p(gof), ctypes.byref(G), ctypes.byref(nc))
    if rc:
        raise MemoryError("oracle group_build failed")
    return gof, int(G.value), int(nc.value)


def cosine_stats(N, rp, ci, v, nsq):
    """Definitions 1-2 at the row level: (nonzero entries of the N x N row-cosine
    table, sum of |cos| over them in units of 2^-32, zn, nn)."""
    rp, ci, v = _csr(rp, ci, v)
    nsq = np.ascontiguousarray(nsq, np.float64)
    nz = ctypes.c_int64(0)
    tot = ctypes.c_uint64(0)
    rc = _load().orc_cosine_stats(ctypes.c_int64(N), _p(rp), _p(ci), _p(v), _p(nsq), ctypes.byref(nz),
                                  ctypes.byref(tot))
    if rc:
        raise MemoryError("oracle cosine_stats failed")
    num = float(N) * float(N)
    return int(nz.value), int(tot.value), (num - nz.value) / num, tot.value * 2.0 ** -32 / num


def group_lists(group_of, G):
    gof = np.ascontiguousarray(group_of, np.int32)
    N = gof.size
    gptr = np.empty(G + 1, np.int64)
    grows = np.empty(max(N, 1), np.int32)
    _load().orc_group_lists(ctypes.c_int64(N), _p(gof), ctypes.c_int64(G), _p(gptr), _p(grows))
    return gptr, grows[: int(gptr[-1])]


def sweep(N, rp, ci, v, nsq, f, gptr, grows, x, nsweeps=1) -> np.ndarray:
    """nsweeps orthogonal-group sweeps (Eq. 3.3 / Algorithm 4); returns the new x."""
    rp, ci, v = _csr(rp, ci, v)
    x = np.array(x, dtype=np.float64, copy=True)
    gptr = np.ascontiguousarray(gptr, np.int64)
    grows = np.ascontiguousarray(grows, np.int32)
    rc = _load().orc_sweep(ctypes.c_int64(N), _p(rp), _p(ci), _p(v),
                           _p(np.ascontiguousarray(nsq, np.float64)),
                           _p(np.ascontiguousarray(f, np.float64)), ctypes.c_int64(gptr.size - 1),
                           _p(gptr), _p(grows), _p(x), ctypes.c_int64(nsweeps))
    if rc:
        raise MemoryError("oracle sweep failed")
    return x


def group_step(rp, ci, v, nsq, f, rows, x) -> np.ndarray:
    """One group projection from x (rows = the group's row list); returns new x."""
    rp, ci, v = _csr(rp, ci, v)
    x = np.array(x, dtype=np.float64, copy=True)
    rows = np.ascontiguousarray(rows, np.int32)
    _load().orc_group_step(_p(rp), _p(ci), _p(v), _p(np.ascontiguousarray(nsq, np.float64)),
                           _p(np.ascontiguousarray(f, np.float64)), _p(rows),
                           ctypes.c_int64(rows.size), _p(x))
    return x


def group_step_pinv(rp, ci, v, nsq, f, rows, x, K) -> np.ndarray:
    """One group step of Eq. 1.3 from x with K Jacobi steps on the group's Gram
    system (K = 0: the simultaneous step); returns the new x."""
    rp, ci, v = _csr(rp, ci, v)
    N = rp.size - 1
    x = np.array(x, dtype=np.float64, copy=True)
    rows = np.ascontiguousarray(rows, np.int32)
    rc = _load().orc_group_step_pinv(ctypes.c_int64(N), _p(rp), _p(ci), _p(v),
                                     _p(np.ascontiguousarray(nsq, np.float64)),
                                     _p(np.ascontiguousarray(f, np.float64)), _p(rows),
                                     ctypes.c_int64(rows.size), _p(x), ctypes.c_int32(K))
    if rc:
        raise MemoryError("oracle group_step_pinv failed")
    return x


def residual(N, rp, ci, v, f, x) -> float:
    rp, ci, v = _csr(rp, ci, v)
    return float(_load().orc_residual(ctypes.c_int64(N), _p(rp), _p(ci), _p(v),
                                      _p(np.ascontiguousarray(f, np.float64)),
                                      _p(np.ascontiguousarray(x, np.float64))))


@dataclasses.dataclass
class Setup:
    N: int
    perm: np.ndarray
    rp: np.ndarray
    ci: np.ndarray
    v: np.ndarray
    f: np.ndarray
    x0: np.ndarray
    nsq: np.ndarray
    group_of: np.ndarray
    G: int
    info: Info


def setup(m, n, rp, ci, v, f, x0=None, thr=0.1) -> Setup:
    """Extend + RCM + permute + norms + groups (everything before the sweeps)."""
    rp, ci, v = _csr(rp, ci, v)
    N = max(m, n)
    nnz = int(rp[-1])
    f = np.ascontiguousarray(f, np.float64)
    x0p = None if x0 is None else np.ascontiguousarray(x0, np.float64)
    perm = np.empty(N, np.int32)
    rpt = np.empty(N + 1, np.int64)
    cit = np.empty(max(nnz, 1), np.int32)
    vt = np.empty(max(nnz, 1), np.float64)
    ft = np.empty(N, np.float64)
    xt = np.empty(N, np.float64)
    nsq = np.empty(N, np.float64)
    gof = np.empty(N, np.int32)
    G = ctypes.c_int64(0)
    info = _Info()
    rc = _load().orc_setup_export(
        ctypes.c_int64(m), ctypes.c_int64(n), _p(rp), _p(ci), _p(v), _p(f),
        None if x0p is None else _p(x0p), ctypes.c_double(thr), _p(perm), _p(rpt), _p(cit),
        _p(vt), _p(ft), _p(xt), _p(nsq), _p(gof), ctypes.byref(G), ctypes.byref(info))
    if rc:
        raise ValueError(f"oracle setup failed ({rc})")
    return Setup(N, perm, rpt, cit[:nnz], vt[:nnz], ft, xt, nsq, gof, int(G.value), _info(info))


def solve(m, n, rp, ci, v, f, x0=None, thr=0.1, tol=1e-8, maxit=10000, check_every=1,
          precision=0, inner_sweeps=4, max_outer=100, stagnation=0.0, return_setup=False, pinv_iters=0):
    """Whole OBK-RCM solve (extend, RCM, groups, sweeps to tol, un-permute).
    pinv_iters > 0: group steps of Eq. 1.3 with that many Jacobi steps (FP64).
    Returns (status, x[n], Info) and, with return_setup, also (perm, group_of)."""
    rp, ci, v = _csr(rp, ci, v)
    N = max(m, n)
    f = np.ascontiguousarray(f, np.float64)
    x0p = None if x0 is None else np.ascontiguousarray(x0, np.float64)
    x = np.empty(n, np.float64)
    perm = np.empty(N, np.int32)
    gof = np.empty(N, np.int32)
    info = _Info()
    opts = _Opts(check_every, precision, inner_sweeps, max_outer, stagnation, pinv_iters, 0)
    st = _load().orc_solve(ctypes.c_int64(m), ctypes.c_int64(n), _p(rp), _p(ci), _p(v), _p(f),
                           None if x0p is None else _p(x0p), ctypes.c_double(thr),
                           ctypes.c_double(tol), ctypes.c_int64(maxit), ctypes.byref(opts),
                           _p(x), ctypes.byref(info), _p(perm), _p(gof))
    if st < 0:
        raise ValueError(f"oracle solve rejected the input ({st})")
    if return_setup:
        return st, x, _info(info), perm, gof
    return st, x, _info(info)


def block_classes(N, rp, ci, v, k, thr):
    """Algorithm 4's classes on k uniform row blocks: (list of Oclass pairs, Nclass list)."""
    rp, ci, v = _csr(rp, ci, v)
    pairs = np.empty(2 * k + 2, np.int32)
    ncl = np.empty(k + 1, np.int32)
    np_ = ctypes.c_int32(0)
    nq = ctypes.c_int32(0)
    rc = _load().orc_block_classes(ctypes.c_int64(N), _p(rp), _p(ci), _p(v), ctypes.c_int32(k),
                                   ctypes.c_double(thr), _p(pairs), ctypes.byref(np_), _p(ncl), ctypes.byref(nq))
    if rc:
        raise MemoryError("oracle block_classes failed")
    return [(int(pairs[2 * i]), int(pairs[2 * i + 1])) for i in range(np_.value)], [int(c) for c in ncl[: nq.value]]


def block_project(rp, ci, v, f, b0, b1, x, inner_max=500, inner_tol=1e-13) -> np.ndarray:
    """x + A_b^+ (f_b - A_b x) for the rows [b0, b1), by CGLS from zero."""
    rp, ci, v = _csr(rp, ci, v)
    N = rp.size - 1
    x = np.array(x, dtype=np.float64, copy=True)
    rc = _load().orc_block_project(ctypes.c_int64(N), _p(rp), _p(ci), _p(v), _p(np.ascontiguousarray(f, np.float64)),
                                   ctypes.c_int64(b0), ctypes.c_int64(b1), _p(x), ctypes.c_int32(inner_max),
                                   ctypes.c_double(inner_tol))
    if rc:
        raise MemoryError("oracle block_project failed")
    return x


def solve_blocks(m, n, rp, ci, v, f, x0=None, k=8, thr=0.1, tol=1e-8, maxit=1000, inner_max=500, inner_tol=1e-13):
    """Algorithm 4 as printed (k uniform blocks, centroid-cosine classes, CGLS
    block projections).  Returns (status, x[n], Info, number of pairs, Nclass size)."""
    rp, ci, v = _csr(rp, ci, v)
    f = np.ascontiguousarray(f, np.float64)
    x0p = None if x0 is None else np.ascontiguousarray(x0, np.float64)
    x = np.empty(n, np.float64)
    info = _Info()
    np_ = ctypes.c_int32(0)
    nq = ctypes.c_int32(0)
    st = _load().orc_solve_blocks(ctypes.c_int64(m), ctypes.c_int64(n), _p(rp), _p(ci), _p(v), _p(f),
                                  None if x0p is None else _p(x0p), ctypes.c_int32(k), ctypes.c_double(thr),
                                  ctypes.c_double(tol), ctypes.c_int64(maxit), ctypes.c_int32(inner_max),
                                  ctypes.c_double(inner_tol), _p(x), ctypes.byref(info), ctypes.byref(np_),
                                  ctypes.byref(nq))
    if st < 0:
        raise ValueError(f"oracle solve_blocks rejected the input ({st})")
    return st, x, _info(info), np_.value, nq.value
