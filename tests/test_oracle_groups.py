"""Pins of the oracle's row norms and cosine-threshold grouping (Section 3.3 at
k = m: cos_ij = (A_i, A_j)/(||A_i|| ||A_j||), conflict when |cos_ij| >= thr,
greedy first-fit groups in index order).

Checked against a dense brute force (numpy A A^T): every pair inside a group is
below the threshold, every row sits in the first group it could join, the
number of conflicting pairs matches, and special cases reduce to known answers
(diagonal -> one group, parallel rows -> all singletons, zero rows skipped).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle_helpers import dense_cos

AMBIG = 1e-12  # pairs this close to thr are decided by rounding; skipped in checks


def test_row_norms_match_exact_sum():
    s = synth.random_dominant(300, seed=11)
    A = s.A
    nsq = oracle.row_norms(A.m, A.row_ptr, A.val)
    for i in range(A.m):
        seg = A.val[A.row_ptr[i]:A.row_ptr[i + 1]]
        exact = math.fsum(float(a) * float(a) for a in seg)
        assert abs(nsq[i] - exact) <= 4 * np.finfo(float).eps * exact


@pytest.mark.parametrize("gen,thr", [
    (lambda: synth.random_dominant(250, seed=21).A, 0.1),
    (lambda: synth.random_dominant(250, seed=22).A, 0.02),
    (lambda: synth.knn_dominant(400, seed=23).A, 0.1),
    (lambda: synth.rect_random(300, 120, 6, seed=24).A, 0.1),
])
def test_groups_against_dense_brute_force(gen, thr):
    A = gen()
    N = max(A.m, A.n)
    rp = np.concatenate([A.row_ptr, np.full(N - A.m, A.row_ptr[-1])]).astype(np.int64)
    Asq = synth.CSR(N, N, rp, A.col_idx, A.val)
    nsq = oracle.row_norms(N, rp, A.val)
    gof, G, nconf = oracle.group_build(N, rp, A.col_idx, A.val, nsq, thr)
    D, C, nrm = dense_cos(Asq)
    zero = nrm == 0
    assert np.all(gof[zero] == -1) and np.all(gof[~zero] >= 0)
    assert G == gof.max() + 1
    absC = np.abs(np.nan_to_num(C))
    conflict = (absC >= thr) & ~np.eye(N, dtype=bool)
    conflict[zero, :] = False
    conflict[:, zero] = False
    clear = np.abs(absC - thr) > AMBIG
    # no conflicting pair shares a group
    same = gof[:, None] == gof[None, :]
    bad = same & conflict & clear & (gof[:, None] >= 0)
    assert not bad.any()
    # first-fit minimality: for every earlier group h < g(i), some earlier row of
    # group h conflicts with row i
    for i in np.flatnonzero(~zero):
        for h in range(gof[i]):
            js = np.flatnonzero((gof[:i] == h))
            assert (conflict[i, js] | ~clear[i, js]).any(), (i, h)
    # conflict count (pairs i > j)
    low = np.tril(conflict, -1)
    n_clear = int((low & clear).sum())
    n_amb = int((np.tril(~clear, -1) & np.tril(~np.eye(N, dtype=bool))).sum())
    assert n_clear <= nconf <= n_clear + n_amb


def test_diagonal_is_one_group():
    N = 50
    A = synth.csr_from_coo(N, N, np.arange(N), np.arange(N), np.arange(1, N + 1, dtype=float))
    nsq = oracle.row_norms(N, A.row_ptr, A.val)
    gof, G, nconf = oracle.group_build(N, A.row_ptr, A.col_idx, A.val, nsq, 0.1)
    assert G == 1 and nconf == 0 and np.all(gof == 0)


def test_parallel_rows_are_singletons():
    N = 6
    rows = np.repeat(np.arange(N), 2)
    cols = np.tile([0, 1], N)
    vals = np.tile([1.0, 2.0], N) * np.repeat(np.arange(1, N + 1), 2)
    A = synth.csr_from_coo(N, N, rows, cols, vals)
    nsq = oracle.row_norms(N, A.row_ptr, A.val)
    gof, G, nconf = oracle.group_build(N, A.row_ptr, A.col_idx, A.val, nsq, 0.5)
    assert gof.tolist() == list(range(N)) and G == N and nconf == N * (N - 1) // 2


def test_negative_cosine_conflicts():
    # rows at cos = -0.9: |cos| is compared, so they must not share a group
    A = synth.csr_from_coo(2, 2, np.array([0, 0, 1, 1]), np.array([0, 1, 0, 1]),
                           np.array([1.0, 0.0, -0.9, math.sqrt(1 - 0.81)]))
    nsq = oracle.row_norms(2, A.row_ptr, A.val)
    gof, G, _ = oracle.group_build(2, A.row_ptr, A.col_idx, A.val, nsq, 0.1)
    assert gof.tolist() == [0, 1]


def test_group_lists_are_ascending_partitions():
    A = synth.random_dominant(300, seed=31).A
    nsq = oracle.row_norms(A.m, A.row_ptr, A.val)
    gof, G, _ = oracle.group_build(A.m, A.row_ptr, A.col_idx, A.val, nsq, 0.1)
    gptr, grows = oracle.group_lists(gof, G)
    assert gptr[0] == 0 and gptr[-1] == A.m
    for g in range(G):
        seg = grows[gptr[g]:gptr[g + 1]]
        assert np.all(np.diff(seg) > 0) and np.all(gof[seg] == g)
