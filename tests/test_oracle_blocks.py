"""Pins of the oracle's paper-literal block form (Section 3.3, Algorithm 4):
the CGLS block projection against the SVD pseudo-inverse, the classes on
matrices whose centroid cosines are known, one block (k = 1) giving the
least-squares solution, and convergence on consistent systems."""
import numpy as np
import pytest

import oracle
import synth


def dense_projection(A, b0, b1, f, x):
    D = A.to_dense()[b0:b1]
    return x + np.linalg.pinv(D) @ (f[b0:b1] - D @ x)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_block_projection_equals_pinv(seed):
    s = synth.random_dominant(60, 4, seed=seed)
    A = s.A
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(60)
    xb = oracle.block_project(A.row_ptr, A.col_idx, A.val, s.f, 10, 35, x)
    xp = dense_projection(A, 10, 35, s.f, x)
    assert np.linalg.norm(xb - xp) / np.linalg.norm(xp) < 1e-12
    # the block's equations hold afterwards
    D = A.to_dense()[10:35]
    assert np.abs(D @ xb - s.f[10:35]).max() < 1e-10


def test_rank_deficient_block_takes_the_minimum_norm_correction():
    # two identical rows in the block (consistent): A_b^+ picks the minimum-norm correction
    n = 12
    rows = [0, 0, 1, 1, 2, 2] + list(range(3, n))
    cols = [0, 5, 0, 5, 3, 7] + list(range(3, n))
    vals = [1.0, 2.0, 1.0, 2.0, 1.5, -1.0] + [1.0] * (n - 3)
    A = synth.csr_from_coo(n, n, np.array(rows), np.array(cols), np.array(vals))
    f = np.ones(n)
    f[1] = f[0]
    x = np.zeros(n)
    xb = oracle.block_project(A.row_ptr, A.col_idx, A.val, f, 0, 3, x)
    xp = dense_projection(A, 0, 3, f, x)
    assert np.linalg.norm(xb - xp) < 1e-12


def test_classes_of_disjoint_blocks():
    # block-diagonal pattern: every pair of block centroids is orthogonal, so the
    # blocks pair up in order and an odd last block is left to Nclass
    k, w = 5, 8
    N = k * w
    r, c, vv = [], [], []
    rng = np.random.default_rng(4)
    for b in range(k):
        for i in range(w):
            row = b * w + i
            for col in rng.choice(w, 3, replace=False):
                r.append(row); c.append(b * w + int(col)); vv.append(rng.uniform(0.5, 1.5))
    A = synth.csr_from_coo(N, N, np.array(r), np.array(c), np.array(vv))
    pairs, ncl = oracle.block_classes(N, A.row_ptr, A.col_idx, A.val, k, 0.1)
    assert pairs == [(0, 1), (2, 3)] and ncl == [4]


def test_classes_of_overlapping_blocks():
    # every row has the same positive entries in the first columns: all
    # centroid cosines are large, no pair forms, Nclass holds every block
    N, k = 40, 4
    r = np.repeat(np.arange(N), 3)
    c = np.tile([0, 1, 2], N)
    vv = np.ones(3 * N)
    A = synth.csr_from_coo(N, N, r, c, vv)
    pairs, ncl = oracle.block_classes(N, A.row_ptr, A.col_idx, A.val, k, 0.1)
    assert pairs == [] and ncl == [0, 1, 2, 3]


def test_one_block_is_least_squares():
    s = synth.rect_random(120, 50, 6, seed=3, noise=1e-2)
    A = s.A
    st, x, info, np_, nq = oracle.solve_blocks(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, k=1, tol=1e-14,
                                               maxit=1, inner_max=2000, inner_tol=1e-15)
    xls = np.linalg.lstsq(A.to_dense(), s.f, rcond=None)[0]
    assert np_ == 0 and nq == 1 and info.sweeps == 1
    assert np.linalg.norm(x - xls) / np.linalg.norm(xls) < 1e-10


@pytest.mark.parametrize("k", [2, 5, 8])
def test_block_form_converges(k):
    s = synth.random_dominant(300, 5, seed=9)
    A = s.A
    st, x, info, np_, nq = oracle.solve_blocks(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, k=k, tol=1e-10,
                                               maxit=2000)
    assert st == 0
    assert np.linalg.norm(x - s.xstar) / np.linalg.norm(s.xstar) < 1e-8
    assert 2 * np_ + nq == k
