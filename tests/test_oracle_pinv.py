"""Pins of the oracle's Eq. 1.3 group step for near-orthogonal groups (Jacobi
steps on the group's Gram system): against the SVD pseudo-inverse projection,
the simultaneous step at K = 0, exactness for orthogonal groups, and a whole
solve."""
import numpy as np
import pytest

import oracle
import synth


def near_orthogonal_group(n_rows=6, ncols=40, seed=0):
    """Rows with one private column each (diagonal-like) plus weak shared
    entries, so that every row's sum of |cos| to the others is below one."""
    rng = np.random.default_rng(seed)
    r, c, v = [], [], []
    for i in range(n_rows):
        r.append(i); c.append(i); v.append(rng.uniform(2.0, 3.0))
        for _ in range(3):
            r.append(i); c.append(int(rng.integers(n_rows, ncols))); v.append(rng.uniform(-0.3, 0.3))
    r, c, v = np.array(r), np.array(c), np.array(v)
    key = r * ncols + c
    _, first = np.unique(key, return_index=True)
    A = synth.csr_from_coo(ncols, ncols, r[first], c[first], v[first])
    return A


def pinv_step(A, rows, f, x):
    D = A.to_dense()
    At = D[rows]
    return x + np.linalg.pinv(At) @ (f[rows] - At @ x)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_converged_jacobi_equals_svd_pinv(seed):
    A = near_orthogonal_group(seed=seed)
    rng = np.random.default_rng(seed + 10)
    nsq = oracle.row_norms(A.m, A.row_ptr, A.val)
    rows = np.arange(6, dtype=np.int32)
    f = rng.standard_normal(A.m)
    x = rng.standard_normal(A.n)
    D = A.to_dense()[:6]
    cosm = np.abs(D @ D.T) / np.sqrt(np.outer(nsq[:6], nsq[:6]))
    assert (cosm.sum(1) - 1.0).max() < 1.0  # Jacobi converges (Gershgorin)
    xk = oracle.group_step_pinv(A.row_ptr, A.col_idx, A.val, nsq, f, rows, x, 200)
    xp = pinv_step(A, rows, f, x)
    assert np.linalg.norm(xk - xp) / np.linalg.norm(xp) < 1e-13
    # after the exact projection the group's residual vanishes
    assert np.abs(D @ xk - f[:6]).max() < 1e-12


def test_zero_iterations_is_the_simultaneous_step():
    A = near_orthogonal_group(seed=5)
    rng = np.random.default_rng(1)
    nsq = oracle.row_norms(A.m, A.row_ptr, A.val)
    rows = np.arange(6, dtype=np.int32)
    f = rng.standard_normal(A.m)
    x = rng.standard_normal(A.n)
    x0 = oracle.group_step_pinv(A.row_ptr, A.col_idx, A.val, nsq, f, rows, x, 0)
    xs = oracle.group_step(A.row_ptr, A.col_idx, A.val, nsq, f, rows, x)
    assert np.array_equal(x0, xs)


def test_orthogonal_group_any_iterations():
    # disjoint columns: the Gram matrix is diagonal, every K gives the same step
    n = 30
    A = synth.csr_from_coo(n, n, np.arange(n), np.arange(n), np.linspace(1.0, 2.0, n))
    nsq = oracle.row_norms(A.m, A.row_ptr, A.val)
    rows = np.arange(0, n, 2, dtype=np.int32)
    rng = np.random.default_rng(2)
    f, x = rng.standard_normal(n), rng.standard_normal(n)
    a = oracle.group_step_pinv(A.row_ptr, A.col_idx, A.val, nsq, f, rows, x, 0)
    b = oracle.group_step_pinv(A.row_ptr, A.col_idx, A.val, nsq, f, rows, x, 7)
    assert np.array_equal(a, b)


def test_solve_with_exact_group_steps():
    s = synth.random_dominant(400, 5, seed=8)
    A = s.A
    st0, x0, i0 = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, tol=1e-10, maxit=5000)
    st1, x1, i1 = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, tol=1e-10, maxit=5000, pinv_iters=8)
    assert st0 == 0 and st1 == 0
    assert np.linalg.norm(x1 - s.xstar) / np.linalg.norm(s.xstar) < 1e-8
    # exact projections need not take fewer sweeps than the simultaneous step
    # (here 49 against 47); the Jacobi steps have converged by K = 8
    st2, x2, i2 = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, tol=1e-10, maxit=5000, pinv_iters=16)
    assert i2.sweeps == i1.sweeps
    assert np.linalg.norm(x2 - x1) / np.linalg.norm(x1) < 1e-12
