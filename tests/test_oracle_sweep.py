"""Pins of the oracle's group projection, sweep, residual and whole solve.

Eq. 1.3 / Eq. 3.3: for a group of mutually orthogonal rows the simultaneous
scaled-residual update equals the pseudo-inverse projection (checked against
numpy's SVD pinv) and zeroes the group's residual.  For near-orthogonal groups
it stays within the Neumann bound rho/(1-rho) of the pinv step (rho = the
largest off-diagonal row sum of the normalised group Gram matrix).
Eq. 3.14-3.15 (Fig. 1): closed forms in two dimensions.  Theorem 1: error
contraction on consistent systems, limit = minimum-norm solution for m < n
(Algorithm 6, Table 10); Algorithm 5: the padded unknowns never move.
Table 4 (bcsstm39, IT = 1): a diagonal system is solved in one sweep.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _orthogonal_group_matrix(seed):
    """8 x 8 matrix whose rows 0..3 are mutually orthogonal (built with QR) and
    whose rows 4..7 are generic; dense storage as CSR."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((8, 8)))
    D = np.vstack([Q[:4] * rng.uniform(0.5, 3.0, size=(4, 1)), rng.standard_normal((4, 8))])
    r, c = np.nonzero(np.ones_like(D))
    return synth.csr_from_coo(8, 8, r, c, D[r, c]), D


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_orthogonal_group_step_equals_pinv_projection(seed):
    A, D = _orthogonal_group_matrix(seed)
    rng = np.random.default_rng(100 + seed)
    f = rng.standard_normal(8)
    x = rng.standard_normal(8)
    nsq = oracle.row_norms(8, A.row_ptr, A.val)
    rows = np.arange(4)
    x1 = oracle.group_step(A.row_ptr, A.col_idx, A.val, nsq, f, rows, x)
    At = D[:4]
    expect = x + np.linalg.pinv(At) @ (f[:4] - At @ x)
    assert np.allclose(x1, expect, rtol=0, atol=1e-14 * max(1.0, np.abs(expect).max()))
    # the group's own residual vanishes after its update
    assert np.abs(f[:4] - At @ x1).max() <= 1e-12 * max(1.0, np.abs(f).max())
    # a dropped term, wrong sign or transposed operand breaks these:
    assert not np.allclose(x1, x)


def test_near_orthogonal_group_within_neumann_bound():
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((10, 10)))
    At = Q[:5] + 0.02 * rng.standard_normal((5, 10))
    D = np.vstack([At, rng.standard_normal((5, 10))])
    r, c = np.nonzero(np.ones_like(D))
    A = synth.csr_from_coo(10, 10, r, c, D[r, c])
    f = rng.standard_normal(10)
    x = rng.standard_normal(10)
    nsq = oracle.row_norms(10, A.row_ptr, A.val)
    x1 = oracle.group_step(A.row_ptr, A.col_idx, A.val, nsq, f, np.arange(5), x)
    U = x1 - x
    P = np.linalg.pinv(At) @ (f[:5] - At @ x)
    nrm = np.linalg.norm(At, axis=1)
    Cn = (At @ At.T) / np.outer(nrm, nrm)
    rho = (np.abs(Cn) - np.eye(5)).sum(axis=1).max()
    assert rho < 1
    assert np.linalg.norm(U - P) <= rho / (1 - rho) * np.linalg.norm(P) + 1e-14
    # the simultaneous update is A^T D^-1 r from the group-start x (not sequential)
    Useq = x.copy()
    for i in range(5):
        Useq = Useq + (f[i] - At[i] @ Useq) / (At[i] @ At[i]) * At[i]
    assert not np.allclose(U, Useq - x, atol=1e-12)


def test_two_dimensional_angle_closed_form():
    # Eq. 3.14-3.15: alternating projections onto two lines at angle theta shrink
    # the error by exactly cos(theta) per projection after the first one
    for theta in (0.3, 0.9, 1.3):
        a1 = np.array([1.0, 0.0])
        a2 = np.array([math.cos(theta), math.sin(theta)])
        D = np.vstack([a1, a2])
        A = synth.csr_from_coo(2, 2, np.array([0, 1, 1]), np.array([0, 0, 1]),
                               np.array([1.0, a2[0], a2[1]]))
        xs = np.array([0.7, -1.1])
        f = D @ xs
        nsq = oracle.row_norms(2, A.row_ptr, A.val)
        x = np.array([3.0, 2.0])
        errs = []
        for k in range(6):
            x = oracle.group_step(A.row_ptr, A.col_idx, A.val, nsq, f, np.array([k % 2]), x)
            errs.append(np.linalg.norm(x - xs))
        ratios = np.array(errs[1:]) / np.array(errs[:-1])
        assert np.allclose(ratios, abs(math.cos(theta)), rtol=1e-12)


def test_orthogonal_2d_exact_in_one_sweep():
    # Fig. 1 right panel: orthogonal hyperplanes reach x* in two projections.  The
    # grouping puts both rows in one group (cos = 0), one sweep solves it.
    A = synth.csr_from_coo(2, 2, np.array([0, 0, 1, 1]), np.array([0, 1, 0, 1]),
                           np.array([2.0, 1.0, -1.0, 2.0]))
    xs = np.array([1.5, -0.5])
    f = A.to_dense() @ xs
    st, x, info = oracle.solve(2, 2, A.row_ptr, A.col_idx, A.val, f, tol=1e-14, maxit=5)
    assert st == oracle.OK and info.sweeps == 1 and info.groups == 1
    assert np.allclose(x, xs, atol=1e-15)


def test_diagonal_system_one_sweep():
    N = 500
    rng = np.random.default_rng(3)
    d = rng.uniform(0.5, 2.0, N)
    A = synth.csr_from_coo(N, N, np.arange(N), np.arange(N), d)
    xs = rng.standard_normal(N)
    st, x, info = oracle.solve(N, N, A.row_ptr, A.col_idx, A.val, d * xs, tol=1e-14, maxit=10)
    assert st == oracle.OK and info.sweeps == 1 and info.groups == 1
    assert np.allclose(x, xs, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("n,seed", [(6, 1), (9, 2), (12, 3)])
def test_small_square_matches_dense_solve(n, seed):
    rng = np.random.default_rng(seed)
    D = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.4) + np.diag(rng.uniform(3, 5, n))
    r, c = np.nonzero(D)
    A = synth.csr_from_coo(n, n, r, c, D[r, c])
    f = rng.standard_normal(n)
    st, x, info = oracle.solve(n, n, A.row_ptr, A.col_idx, A.val, f, tol=1e-13, maxit=100000)
    assert st == oracle.OK
    assert np.allclose(x, np.linalg.solve(D, f), rtol=1e-10, atol=1e-11)


def test_error_contracts_per_group_and_linearly():
    s = synth.random_dominant(400, seed=5)
    A = s.A
    su = oracle.setup(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1)
    gptr, grows = oracle.group_lists(su.group_of, su.G)
    xs_t = s.xstar[su.perm]
    x = su.x0.copy()
    errs = [np.linalg.norm(x - xs_t)]
    per_sweep = []
    for sw in range(12):
        for g in range(su.G):
            x = oracle.group_step(su.rp, su.ci, su.v, su.nsq, su.f, grows[gptr[g]:gptr[g + 1]], x)
            errs.append(np.linalg.norm(x - xs_t))
        per_sweep.append(errs[-1])
    assert np.all(np.diff(errs) <= 1e-12 * errs[0])
    slope = np.polyfit(np.arange(len(per_sweep)), np.log(per_sweep), 1)[0]
    assert slope < -0.1
    # Eq. 3.4: the error is the same in the permuted and original orderings
    xo = np.empty_like(x)
    xo[su.perm] = x
    assert math.isclose(np.linalg.norm(xo - s.xstar), errs[-1], rel_tol=1e-14)


def test_underdetermined_gives_minimum_norm_solution():
    # Algorithm 6 / Table 10: with x0 = 0 the iterates stay in range(A^T)
    s = synth.rect_random(40, 100, 8, seed=9)
    A = s.A
    st, x, info = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, tol=1e-12,
                               maxit=200000)
    assert st == oracle.OK
    D = A.to_dense()
    xmn = np.linalg.pinv(D) @ s.f
    assert np.linalg.norm(x - xmn) <= 1e-9 * np.linalg.norm(xmn)


def test_overdetermined_consistent_and_padding_untouched():
    # Algorithm 5: A^ = [A, O]; the padded unknowns have empty columns and stay 0
    s = synth.rect_random(300, 100, 8, seed=10)
    A = s.A
    st, x, info = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, tol=1e-11,
                               maxit=200000)
    assert st == oracle.OK
    assert np.linalg.norm(x - s.xstar) <= 1e-8 * np.linalg.norm(s.xstar)
    su = oracle.setup(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1)
    gptr, grows = oracle.group_lists(su.group_of, su.G)
    xt = oracle.sweep(su.N, su.rp, su.ci, su.v, su.nsq, su.f, gptr, grows, su.x0, 3)
    xh = np.empty_like(xt)
    xh[su.perm] = xt
    assert np.all(xh[A.n:] == 0.0)


def test_inconsistent_stagnates_not_converged():
    s = synth.rect_random(600, 200, 8, seed=12, noise=1e-3)
    A = s.A
    st, x, info = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, tol=1e-8,
                               maxit=20000, stagnation=1e-12)
    assert st == oracle.NOT_CONVERGED and info.sweeps < 20000
    # the floor is near the least-squares residual, well above tol
    D = A.to_dense()
    xls = np.linalg.lstsq(D, s.f, rcond=None)[0]
    rls = np.linalg.norm(s.f - D @ xls) / np.linalg.norm(s.f)
    assert rls <= info.rel_res < 50 * rls


def test_residual_matches_numpy():
    s = synth.random_dominant(300, seed=13)
    A = s.A
    x = np.random.default_rng(1).standard_normal(300)
    rr = oracle.residual(300, A.row_ptr, A.col_idx, A.val, s.f, x)
    D = A.to_dense()
    assert math.isclose(rr, np.linalg.norm(s.f - D @ x) / np.linalg.norm(s.f), rel_tol=1e-13)


def test_precision_form_reaches_1e10_and_matches_fp64():
    s = synth.random_dominant(1500, seed=14)
    A = s.A
    st64, x64, i64 = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, tol=1e-10,
                                  maxit=10000)
    st, x, info = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, tol=1e-10,
                               maxit=10000, precision=1, inner_sweeps=6)
    assert st64 == oracle.OK and st == oracle.OK
    assert info.rel_res <= 1e-10 and info.outer_iters >= 2
    assert np.linalg.norm(x - x64) <= 1e-8 * np.linalg.norm(x64)


def test_refinement_step_gains_fp32_precision_on_diagonal_system():
    """Pin of the precision form's outer step against what the arithmetic
    fixes.  For a diagonal A every row is one group, so one FP32 sweep solves
    A d = r / beta up to FP32 rounding: the right-hand side (float)(r / beta),
    the FP32 inverse norm and the product each carry a relative error of at
    most 2^-24, so after x += beta d the new residual is at most about
    4 * 2^-24 of the old one, until the FP64 floor (~1e-16).  A residual or a
    correction accumulated in FP32 would stall near 1e-7; a dropped beta or a
    wrong sign would not contract at all."""
    rng = np.random.default_rng(15)
    n = 4000
    d = rng.uniform(0.5, 3.0, n) * rng.choice([-1.0, 1.0], n)
    A = synth.csr_from_coo(n, n, np.arange(n), np.arange(n), d)
    f = d * rng.standard_normal(n)
    rr = [1.0]
    for outer in (1, 2, 3):
        st, x, info = oracle.solve(n, n, A.row_ptr, A.col_idx, A.val, f, tol=1e-300, maxit=100, precision=1,
                                   inner_sweeps=1, max_outer=outer)
        assert info.outer_iters == outer and info.sweeps == outer
        rr.append(info.rel_res)
    bound = 4 * 2.0 ** -24
    assert rr[1] <= bound, rr
    assert rr[2] <= max(bound * rr[1], 1e-15), rr
    assert rr[3] <= 1e-15, rr
    assert np.linalg.norm(x - f / d) <= 1e-15 * np.linalg.norm(f / d)


def test_validate_rejects_bad_csr():
    rp = np.array([0, 2, 3], np.int64)
    assert oracle.validate(2, 2, rp, np.array([0, 1, 1], np.int32), np.ones(3)) == 0
    assert oracle.validate(2, 2, rp, np.array([1, 0, 1], np.int32), np.ones(3)) != 0  # unsorted
    assert oracle.validate(2, 2, rp, np.array([0, 2, 1], np.int32), np.ones(3)) != 0  # range
    assert oracle.validate(2, 2, rp, np.array([0, 1, 1], np.int32),
                           np.array([1.0, np.nan, 1.0])) != 0
    assert oracle.validate(2, 2, np.array([0, 3, 2]), np.array([0, 1, 1], np.int32),
                           np.ones(3)) != 0


def test_adaptive_check_schedule_never_stops_early():
    # the adaptive cadence only moves residual checks; it must never report
    # convergence before the every-sweep test would, and overshoots little
    s = synth.knn_dominant(20000, seed=41)
    A = s.A
    for tol in (1e-6, 1e-8, 1e-10):
        _, _, fixed = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, tol=tol, maxit=5000, check_every=1)
        st, _, ad = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, tol=tol, maxit=5000, check_every=-1)
        assert st == oracle.OK and ad.rel_res <= tol
        assert fixed.sweeps <= ad.sweeps <= fixed.sweeps + max(2, fixed.sweeps // 4)


def test_all_zero_matrix():
    """The degenerate empty matrix: every vertex is its own component, so the
    order is the identity reversed; no row joins a group; f = 0 is solved at
    once by x = 0 and f != 0 cannot be reached."""
    m = n = 5
    rp = np.zeros(m + 1, np.int64)
    ci = np.zeros(0, np.int32)
    v = np.zeros(0)
    su = oracle.setup(m, n, rp, ci, v, np.zeros(m), thr=0.1)
    assert su.G == 0 and np.array_equal(su.perm, np.arange(m)[::-1])
    st, x, info = oracle.solve(m, n, rp, ci, v, np.zeros(m), thr=0.1, tol=1e-8, maxit=10)
    assert st == 0 and info.sweeps == 0 and not x.any()
    st, x, info = oracle.solve(m, n, rp, ci, v, np.ones(m), thr=0.1, tol=1e-8, maxit=10)
    assert st == 1 and not x.any()
