"""The seeded generators return valid CSR systems of the stated shapes, reproducibly."""
import numpy as np

import oracle
import synth


def _valid(A):
    return oracle.validate(A.m, A.n, A.row_ptr, A.col_idx, A.val) == 0


def test_random_dominant_shape_and_dominance():
    s = synth.random_dominant(500, 7, seed=1)
    A = s.A
    assert _valid(A) and A.nnz == 500 * 8
    D = A.to_dense()
    off = np.abs(D).sum(axis=1) - np.abs(np.diag(D))
    assert np.allclose(np.diag(D), 1 + off)
    assert np.allclose(A.matvec(s.xstar), s.f)


def test_knn_symmetric_pattern_and_diagonal():
    s = synth.knn_dominant(2000, 12, seed=2)
    A = s.A
    assert _valid(A)
    D = A.to_dense()
    assert np.array_equal(D != 0, (D != 0).T)
    off = np.abs(D).sum(axis=1) - np.abs(np.diag(D))
    assert np.allclose(np.diag(D), 1.2 * off)
    deg = np.diff(A.row_ptr) - 1
    assert deg.min() >= 12 and 13 <= deg.mean() <= 20


def test_rect_random_no_empty_columns_and_noise():
    s = synth.rect_random(400, 100, 10, seed=3)
    A = s.A
    assert _valid(A) and np.all(np.diff(A.row_ptr) == 10)
    assert np.bincount(A.col_idx, minlength=100).min() > 0
    s2 = synth.rect_random(400, 100, 10, seed=3, noise=1e-3)
    assert 0 < np.linalg.norm(s2.f - s.f) < 1.0


def test_determinism():
    a, b = synth.knn_dominant(1000, seed=9), synth.knn_dominant(1000, seed=9)
    assert np.array_equal(a.A.col_idx, b.A.col_idx) and np.array_equal(a.A.val, b.A.val)
    assert np.array_equal(a.f, b.f)


def test_request_stream_mix():
    reqs = synth.request_stream(400, seed=5, materialize=False)
    ns = np.array([r.n for r in reqs])
    assert ns.min() >= 1000 and ns.max() <= 200000
    over = np.mean([r.m == 2 * r.n for r in reqs])
    assert 0.15 < over < 0.35
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) >= 0)


def test_request_stream_underdetermined_share():
    base = synth.request_stream(400, seed=5, materialize=False)
    mixed = synth.request_stream(400, seed=5, materialize=False, frac_under=0.2)
    # the draw for underdetermined requests leaves the default stream unchanged
    assert [(r.n, r.m, r.precision) for r in base] == [
        (r.n, r.m if r.m >= r.n else r.n, r.precision) for r in mixed]
    under = np.mean([r.m < r.n for r in mixed])
    assert 0.12 < under < 0.28
    assert all(r.m == r.n // 2 for r in mixed if r.m < r.n)
    small = synth.request_stream(30, seed=9, n_lo=1000, n_hi=3000, frac_under=0.5)
    for r in small:
        if r.m < r.n:
            assert r.system.A.m == r.m and r.system.A.n == r.n
