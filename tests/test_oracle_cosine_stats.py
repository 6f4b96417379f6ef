"""Pins of the oracle's cosine-table statistics (Section 3.6, Definitions 1
and 2, at the row level): brute force from the dense normalised A A^T on
integer matrices (every dot product exact, so the counts and the fixed-point
sums must agree exactly), closed forms, and a tolerance check on a real
matrix."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def brute(A):
    """nonzero entries and sum of round(|cos| 2^32) of the N x N row-cosine table."""
    D = A.to_dense()
    N = D.shape[0]
    G = D @ D.T
    nsq = np.diag(G).copy()
    s = np.sqrt(nsq)
    nz, tot = 0, 0
    for i in range(N):
        if nsq[i] == 0.0:
            continue
        nz += 1
        tot += 1 << 32
        for j in range(N):
            if j == i or nsq[j] == 0.0:
                continue
            c = G[i, j] / (s[min(i, j)] * s[max(i, j)])
            if c != 0.0:
                nz += 1
                tot += int(np.rint(abs(c) * 2.0 ** 32))
    return nz, tot


def stats(A):
    nsq = oracle.row_norms(A.m, A.row_ptr, A.val)
    return oracle.cosine_stats(A.m, A.row_ptr, A.col_idx, A.val, nsq)


def int_matrix(n, k, seed, zero_rows=()):
    rng = np.random.default_rng(seed)
    r, c = [], []
    for i in range(n):
        if i in zero_rows:
            continue
        cols = rng.choice(n, k, replace=False)
        r += [i] * k
        c += list(cols)
    v = rng.integers(-3, 4, len(r)).astype(np.float64)
    v[v == 0] = 1.0
    return synth.csr_from_coo(n, n, np.array(r), np.array(c), v)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_against_brute_force(seed):
    A = int_matrix(60, 4, seed, zero_rows=(5, 17))
    nz, tot, zn, nn = stats(A)
    bnz, btot = brute(A)
    assert nz == bnz and tot == btot
    assert zn == pytest.approx((60 * 60 - bnz) / 3600.0, rel=0, abs=1e-15)
    assert nn == pytest.approx(btot * 2.0 ** -32 / 3600.0, rel=1e-15)


def test_identity_closed_form():
    n = 50
    A = synth.csr_from_coo(n, n, np.arange(n), np.arange(n), np.linspace(1, 3, n))
    nz, tot, zn, nn = stats(A)
    assert nz == n and tot == n << 32
    assert zn == pytest.approx(1 - 1 / n) and nn == pytest.approx(1 / n)


def test_parallel_rows_closed_form():
    # every row a multiple of the same vector: |cos| = 1 everywhere
    n = 20
    rows = np.repeat(np.arange(n), 3)
    cols = np.tile([2, 7, 11], n)
    vals = np.repeat(np.arange(1, n + 1, dtype=np.float64), 3) * np.tile([1.0, -2.0, 0.5], n)
    A = synth.csr_from_coo(n, n, rows, cols, vals)
    nz, tot, zn, nn = stats(A)
    assert nz == n * n and zn == 0.0
    assert abs(tot - (n * n << 32)) <= n * n  # each |cos| within one unit of 2^-32 of 1
    assert nn == pytest.approx(1.0, abs=1e-8)


def test_real_matrix_within_rounding():
    s = synth.random_dominant(80, 5, seed=3)
    nz, tot, zn, nn = stats(s.A)
    bnz, btot = brute(s.A)
    assert nz == bnz
    assert abs(tot - btot) <= nz  # fold order may move each |cos| by one unit
