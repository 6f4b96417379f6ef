"""Seeded synthetic inputs for OBK-RCM workloads.

This module only *creates* inputs: sparse matrices in CSR form, exact
solutions x*, right-hand sides f and request streams.  It holds none of the
method's arithmetic (no reordering, grouping or projection); the CUDA path and
the CPU oracle both read what it returns.

The paper measures on SuiteSparse matrices and on MATLAB ``sprandn`` matrices
with unpublished seeds (Section 3.5, Section 4.3); neither is available here,
so these generators stand in for them with the shapes the paper describes:
scattered sparse patterns that RCM turns into a band.

All generators are deterministic functions of their arguments (numpy PCG64).
CSR convention everywhere: ``row_ptr`` int64 [m+1], ``col_idx`` int32 [nnz]
(0-based, strictly increasing inside a row), ``val`` float64 [nnz].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "CSR",
    "System",
    "random_dominant",
    "knn_dominant",
    "rect_random",
    "request_stream",
    "Request",
    "csr_from_coo",
]


@dataclasses.dataclass
class CSR:
    m: int
    n: int
    row_ptr: np.ndarray  # int64 [m+1]
    col_idx: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.m, self.n))
        for i in range(self.m):
            s, e = self.row_ptr[i], self.row_ptr[i + 1]
            d[i, self.col_idx[s:e]] = self.val[s:e]
        return d

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """y = A x, used only to build right-hand sides (f = A x*)."""
        import scipy.sparse as sp

        a = sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.m, self.n))
        return a @ x


@dataclasses.dataclass
class System:
    A: CSR
    xstar: np.ndarray  # float64 [n]
    f: np.ndarray  # float64 [m]
    name: str = ""


def csr_from_coo(m: int, n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    """Build a CSR with sorted, unique columns from COO triplets (no duplicates allowed)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    order = np.argsort(rows * np.int64(max(n, 1)) + cols, kind="stable")
    rows, cols, vals = rows[order], cols[order], np.asarray(vals, dtype=np.float64)[order]
    if rows.size > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if dup.any():
            raise ValueError("duplicate (row, col) entries")
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(m, n, row_ptr, cols.astype(np.int32), vals.copy())


def _distinct_columns(rng: np.random.Generator, m: int, n: int, k: int, skip_diag: bool) -> np.ndarray:
    """k distinct uniform random columns per row, sorted; the diagonal is excluded if asked."""
    pool = n - 1 if skip_diag else n
    if k > pool:
        raise ValueError("k larger than the number of admissible columns")
    rows = np.arange(m, dtype=np.int64)[:, None]
    cols = np.empty((m, k), dtype=np.int64)
    todo = np.arange(m)
    while todo.size:
        c = rng.integers(0, pool, size=(todo.size, k))
        if skip_diag:
            c = c + (c >= rows[todo])
        c.sort(axis=1)
        ok = ~np.any(c[:, 1:] == c[:, :-1], axis=1) if k > 1 else np.ones(todo.size, bool)
        cols[todo[ok]] = c[ok]
        todo = todo[~ok]
    return cols


def random_dominant(n: int, k: int = 7, seed: int = 1000) -> System:
    """Square n x n: each row has k off-diagonal nonzeros at uniform random distinct
    columns with N(0,1) values and diagonal 1 + sum|off-diagonals|; x* ~ N(0,1),
    f = A x*.  (Small square workload, n = 2000 in the paper-sized case.)"""
    rng = np.random.Generator(np.random.PCG64(seed))
    off = _distinct_columns(rng, n, n, k, skip_diag=True)
    offv = rng.standard_normal((n, k))
    diag = 1.0 + np.abs(offv).sum(axis=1)
    rows = np.repeat(np.arange(n), k + 1)
    cols = np.concatenate([off, np.arange(n)[:, None]], axis=1).ravel()
    vals = np.concatenate([offv, diag[:, None]], axis=1).ravel()
    A = csr_from_coo(n, n, rows, cols, vals)
    xstar = rng.standard_normal(n)
    return System(A, xstar, A.matvec(xstar), f"random_dominant(n={n},k={k},seed={seed})")


def _knn(points: np.ndarray, k: int) -> np.ndarray:
    from scipy.spatial import cKDTree

    tree = cKDTree(points)
    _, idx = tree.query(points, k=k + 1, workers=-1)
    n = points.shape[0]
    # drop the point itself (distance 0); fall back to dropping the last
    # neighbour if a duplicate point displaced it
    self_col = idx == np.arange(n)[:, None]
    keep = ~self_col
    no_self = ~self_col.any(axis=1)
    keep[no_self, -1] = False
    return idx[keep].reshape(n, k)


def knn_dominant(n: int, k: int = 12, seed: int = 1001, diag_factor: float = 1.2) -> System:
    """Square n x n with the symmetrised k-nearest-neighbour pattern of n points
    uniform in the unit cube; off-diagonals N(0,1) drawn independently per stored
    entry, diagonal = diag_factor * sum|off-diagonals|.  The vertices are then
    relabelled by a seeded random permutation (the same on rows and columns, so the
    diagonal is kept) to scatter the pattern before RCM.  x* ~ N(0,1), f = A x*."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.random((n, 3))
    nb = _knn(pts, k)
    i = np.repeat(np.arange(n, dtype=np.int64), k)
    j = nb.ravel().astype(np.int64)
    key = np.concatenate([i * n + j, j * n + i])
    key.sort()
    key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    r, c = key // n, key % n
    offv = rng.standard_normal(key.size)
    diag = diag_factor * np.bincount(r, weights=np.abs(offv), minlength=n)
    relabel = rng.permutation(n).astype(np.int64)  # new label of old vertex v
    rows = np.concatenate([relabel[r], relabel])
    cols = np.concatenate([relabel[c], relabel])
    vals = np.concatenate([offv, diag])
    A = csr_from_coo(n, n, rows, cols, vals)
    xstar = rng.standard_normal(n)
    return System(A, xstar, A.matvec(xstar), f"knn_dominant(n={n},k={k},seed={seed})")


def rect_random(m: int, n: int, k: int = 10, seed: int = 1002, noise: float = 0.0,
                full_columns: bool | None = None) -> System:
    """m x n with k distinct uniform random columns per row, N(0,1) values.  For
    m >= n (or full_columns=True) the pattern is redrawn until every column holds a
    nonzero, which makes full column rank near-certain for m >= 2n.  f = A x*
    (+ noise * N(0,1) for the inconsistent variant)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if full_columns is None:
        full_columns = m >= n
    for _ in range(64):
        cols = _distinct_columns(rng, m, n, k, skip_diag=False)
        if not full_columns or np.bincount(cols.ravel(), minlength=n).min() > 0:
            break
    else:  # pragma: no cover - astronomically unlikely for the sizes used
        raise RuntimeError("could not draw a matrix without empty columns")
    vals = rng.standard_normal((m, k))
    A = csr_from_coo(m, n, np.repeat(np.arange(m), k), cols.ravel(), vals.ravel())
    xstar = rng.standard_normal(n)
    f = A.matvec(xstar)
    if noise:
        f = f + noise * rng.standard_normal(m)
    return System(A, xstar, f, f"rect_random(m={m},n={n},k={k},seed={seed},noise={noise})")


@dataclasses.dataclass
class Request:
    index: int
    arrival_s: float
    system: System | None
    n: int
    m: int
    precision: int  # 0 = FP64, 1 = FP32 inner sweeps + FP64 refinement
    seed: int


def request_stream(count: int = 4096, rate_per_s: float = 1000.0, seed: int = 1004,
                   n_lo: int = 1000, n_hi: int = 200_000, frac_over: float = 0.25,
                   materialize: bool = True, frac_under: float = 0.0) -> list[Request]:
    """Poisson arrivals of independent systems.  n is log-uniform in [n_lo, n_hi];
    a fraction frac_over is overdetermined (m = 2n, rect_random recipe), a fraction
    frac_under underdetermined (m = n // 2, rect_random recipe without the
    every-column rule), the rest square (random_dominant recipe).  Precision is
    drawn 50/50 per request.  Request r uses seed 10**6 + r for its system; the
    stream with frac_under = 0 does not depend on that draw."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps) - gaps[0]
    logn = rng.uniform(math.log(n_lo), math.log(n_hi), size=count)
    over = rng.random(count) < frac_over
    prec = (rng.random(count) < 0.5).astype(int)
    under_u = rng.random(count)
    under = ~over & (under_u < frac_under / max(1.0 - frac_over, 1e-12))
    out = []
    for r in range(count):
        n = int(math.floor(math.exp(logn[r])))
        s = 10**6 + r
        if over[r]:
            m = 2 * n
            sys_ = rect_random(m, n, 10, s) if materialize else None
        elif under[r]:
            m = max(n // 2, 1)
            sys_ = rect_random(m, n, 10, s, full_columns=False) if materialize else None
        else:
            m = n
            sys_ = random_dominant(n, 7, s) if materialize else None
        out.append(Request(r, float(t[r]), sys_, n, m, int(prec[r]), s))
    return out
