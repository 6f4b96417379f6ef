"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Permutation, row norms and groups must match bit for bit; the FP64 solve must
match x to ||x_gpu - x_oracle|| / ||x_oracle|| <= 1e-9 after the same number
of sweeps, and stop within one sweep of the oracle.  Cases span several
thread blocks and ragged tails, plus the degenerate inputs of the method.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle_helpers import graph_matrix

pytestmark = pytest.mark.gpu

XTOL = 1e-9  # FP64 parity bound on the relative 2-norm difference of x


@pytest.fixture(scope="module")
def obk():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_00672_gb300 as m

    return m


def _diag(n=777):
    rng = np.random.default_rng(3)
    d = rng.uniform(0.5, 2.0, n)
    A = synth.csr_from_coo(n, n, np.arange(n), np.arange(n), d)
    xs = rng.standard_normal(n)
    return synth.System(A, xs, d * xs, "diag")


def _components():
    # two random components, isolated vertices, and a path; diagonal everywhere
    rng = np.random.default_rng(11)
    N = 900
    edges = set()
    for lo, hi in ((0, 400), (400, 700)):
        for _ in range(3 * (hi - lo)):
            a, b = rng.integers(lo, hi, 2)
            if a != b:
                edges.add((int(min(a, b)), int(max(a, b))))
    for k in range(800, 899):
        edges.add((k, k + 1))
    lab = rng.permutation(N)
    A = graph_matrix(N, [(int(lab[a]), int(lab[b])) for a, b in sorted(edges)])
    vals = rng.standard_normal(A.nnz)
    rows = np.repeat(np.arange(N), np.diff(A.row_ptr))
    vals[rows == A.col_idx] = 0.0
    offs = np.bincount(rows, weights=np.abs(vals), minlength=N)
    vals[rows == A.col_idx] = 1.0 + offs
    A.val = vals
    xs = rng.standard_normal(N)
    return synth.System(A, xs, A.matvec(xs), "components")


def _zero_rows():
    s = synth.random_dominant(500, 5, seed=77)
    A = s.A
    # blank out some rows entirely (explicit zeros) -> they take no part
    v = A.val.copy()
    for i in (0, 17, 250, 499):
        v[A.row_ptr[i]:A.row_ptr[i + 1]] = 0.0
    A.val = v
    f = A.matvec(s.xstar)
    return synth.System(A, s.xstar, f, "zero_rows")


def _hubs():
    # sparse diagonally dominant rows plus three hub rows/columns of degree 2000,
    # 2000 and 2600: heavy frontier vertices in the RCM kernels, slices whose rows
    # differ in length by two orders of magnitude, and segment sorts of every
    # size class (the last hub's lists exceed one block's 2048)
    rng = np.random.default_rng(21)
    N = 6000
    rows, cols = [], []
    for i in range(N):
        c = rng.choice(N - 1, 5, replace=False)
        c[c >= i] += 1
        rows += [i] * 5
        cols += list(c)
    for h, deg in ((17, 2000), (3001, 2000), (5998, 2600)):
        nb = rng.choice(N, deg, replace=False)
        nb = nb[nb != h]
        rows += [h] * len(nb) + list(nb)
        cols += list(nb) + [h] * len(nb)
    r = np.array(rows, np.int64)
    c = np.array(cols, np.int64)
    key = np.unique(r * N + c)
    r, c = key // N, key % N
    v = rng.standard_normal(len(r))
    # weak hub couplings keep every group step contractive (the sum of a hub
    # row's cosines with its group stays below one)
    hub = np.isin(r, (17, 3001, 5998)) | np.isin(c, (17, 3001, 5998))
    v[hub] *= 1e-3
    off = np.bincount(r, weights=np.abs(v), minlength=N)
    r = np.concatenate([r, np.arange(N)])
    c = np.concatenate([c, np.arange(N)])
    v = np.concatenate([v, 1.0 + off])
    A = synth.csr_from_coo(N, N, r, c, v)
    xs = rng.standard_normal(N)
    return synth.System(A, xs, A.matvec(xs), "hubs")


def _many_groups():
    # 150 rows sharing one strong column conflict pairwise (|cos| = 0.41), so
    # first fit needs more than 64 groups
    rng = np.random.default_rng(5)
    N = 1000
    base = synth.random_dominant(N, 3, seed=55).A
    r = np.repeat(np.arange(N), np.diff(base.row_ptr)).astype(np.int64)
    c = base.col_idx.astype(np.int64)
    v = base.val.copy()
    keep = ~((r < 150) & (c == N - 1))
    r, c, v = r[keep], c[keep], v[keep]
    v[(r < 150) & (r == c)] = 12.0
    v[(r < 150) & (r != c)] = 0.0
    r = np.concatenate([r, np.arange(150)])
    c = np.concatenate([c, np.full(150, N - 1)])
    v = np.concatenate([v, np.full(150, 10.0)])
    v[(r == N - 1) & (c == N - 1)] = 2000.0
    A = synth.csr_from_coo(N, N, r, c, v)
    xs = rng.standard_normal(N)
    return synth.System(A, xs, A.matvec(xs), "many_groups")


def _grid_coo(H, W, rng, offset=0):
    # 5-point pattern on an H x W grid, row-major numbering, off-diagonals N(0,1)
    idx = np.arange(H * W).reshape(H, W)
    pairs = [(idx[:, :-1].ravel(), idx[:, 1:].ravel()), (idx[:-1, :].ravel(), idx[1:, :].ravel())]
    r = np.concatenate([a for a, b in pairs] + [b for a, b in pairs]) + offset
    c = np.concatenate([b for a, b in pairs] + [a for a, b in pairs]) + offset
    return r, c, rng.standard_normal(len(r))


def _dominant(N, r, c, v, rng, name):
    off = np.bincount(r, weights=np.abs(v), minlength=N)
    r = np.concatenate([r, np.arange(N)])
    c = np.concatenate([c, np.arange(N)])
    v = np.concatenate([v, 1.0 + off])
    A = synth.csr_from_coo(N, N, r, c, v)
    xs = rng.standard_normal(N)
    return synth.System(A, xs, A.matvec(xs), name)


def _grid2d():
    # 90 x 90 grid: the search starts at a corner, its candidate (the opposite
    # corner) is no farther, so the root stays; 179 BFS levels
    rng = np.random.default_rng(31)
    r, c, v = _grid_coo(90, 90, rng)
    return _dominant(90 * 90, r, c, v, rng, "grid2d")


def _knn_and_grid():
    # two components with long level structures: a kNN graph whose root moves
    # to its first candidate and a 70 x 70 grid whose root stays
    rng = np.random.default_rng(32)
    k = synth.knn_dominant(20000, 12, seed=33).A
    kr = np.repeat(np.arange(k.m), np.diff(k.row_ptr)).astype(np.int64)
    kc = k.col_idx.astype(np.int64)
    off = kr != kc
    gr, gc, gv = _grid_coo(70, 70, rng, offset=k.m)
    N = k.m + 70 * 70
    r = np.concatenate([kr[off], gr])
    c = np.concatenate([kc[off], gc])
    v = np.concatenate([k.val[off], gv])
    return _dominant(N, r, c, v, rng, "knn_and_grid")


CASES = {
    "random_dominant_2000": lambda: synth.random_dominant(2000, 7, seed=1000),
    "knn_30000": lambda: synth.knn_dominant(30000, 12, seed=1001),
    "rect_over_3000x1000": lambda: synth.rect_random(3000, 1000, 10, seed=1002),
    "rect_under_400x1000": lambda: synth.rect_random(400, 1000, 8, seed=7, full_columns=False),
    "diag": _diag,
    "components": _components,
    "zero_rows": _zero_rows,
    "tiny_3x3": lambda: synth.random_dominant(3, 1, seed=5),
    "hubs": _hubs,
    "many_groups": _many_groups,
    "grid2d_90x90": _grid2d,
    "knn_and_grid": _knn_and_grid,
}

_cache = {}


def _case(name):
    if name not in _cache:
        s = CASES[name]()
        A = s.A
        su = oracle.setup(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1)
        _cache[name] = (s, su)
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_setup_bit_exact(obk, name):
    s, su = _case(name)
    A = s.A
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        assert h.N == su.N and h.G == su.G
        assert np.array_equal(h.perm(), su.perm)
        assert np.array_equal(h.row_norms().view(np.uint64), su.nsq.view(np.uint64))
        assert np.array_equal(h.groups(), su.group_of)
        info = h.info()
        assert info.bandwidth_after == su.info.bandwidth_after
        assert info.bandwidth_before == su.info.bandwidth_before
        assert info.n_conflicts == su.info.n_conflicts


def test_setup_symmetric_pattern_with_missing_diagonals(obk):
    # a structurally symmetric pattern (a 60 x 60 grid plus a kNN block) whose
    # rows 0, 3, 6, ... hold no diagonal entry: the RCM graph of such a pattern
    # is each row without its diagonal, taken without the merge with the
    # transpose; an asymmetric copy (one extra entry) takes the merge
    rng = np.random.default_rng(41)
    r, c, v = _grid_coo(60, 60, rng)
    N = 60 * 60
    keep_diag = np.arange(N) % 3 != 0
    d = np.arange(N)[keep_diag]
    r = np.concatenate([r, d])
    c = np.concatenate([c, d])
    v = np.concatenate([v, 4.0 + rng.random(len(d))])
    for extra in (False, True):
        rr, cc, vv = r, c, v
        if extra:
            rr = np.concatenate([r, [5]])
            cc = np.concatenate([c, [N - 7]])
            vv = np.concatenate([v, [0.5]])
        A = synth.csr_from_coo(N, N, rr, cc, vv)
        f = A.matvec(rng.standard_normal(N))
        su = oracle.setup(A.m, A.n, A.row_ptr, A.col_idx, A.val, f, thr=0.1)
        with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
            assert np.array_equal(h.perm(), su.perm)
            assert np.array_equal(h.groups(), su.group_of)
            assert h.info().bandwidth_after == su.info.bandwidth_after


def _pair_cosine(rp, ci, v, nsq, i, j):
    # RN(dot / RN(s_j s_i)), dot the left fold of the products over the columns
    # rows i and j share, ascending (Sec. 3.3 cosine, the oracle's rounding)
    a, ae, b, be = int(rp[i]), int(rp[i + 1]), int(rp[j]), int(rp[j + 1])
    acc = 0.0
    while a < ae and b < be:
        if ci[a] == ci[b]:
            acc = acc + float(v[a]) * float(v[b])
            a += 1
            b += 1
        elif ci[a] < ci[b]:
            a += 1
        else:
            b += 1
    return acc / (math.sqrt(float(nsq[j])) * math.sqrt(float(nsq[i])))


def test_conflicts_at_exact_pair_cosines(obk):
    # thresholds equal to the cosine of an actual pair (and the doubles next to
    # it) put that pair exactly on the decision boundary, where no bound on a
    # lower-precision dot product can decide and the exact FP64 fold must
    s = synth.knn_dominant(3000, 12, seed=1009)
    A = s.A
    base = oracle.setup(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1)
    rp, ci, v, nsq = base.rp, base.ci, base.v, base.nsq
    rng = np.random.default_rng(3)
    picked = []
    for i in rng.permutation(np.arange(200, base.N)):
        cand = set()
        for c in ci[rp[i]:rp[i + 1]]:
            cand.update(int(j) for j in ci[rp[c]:rp[c + 1]] if j < i)
        for j in sorted(cand):
            t = abs(_pair_cosine(rp, ci, v, nsq, int(i), j))
            if 0.02 <= t <= 0.6:
                picked.append(t)
                break
        if len(picked) == 4:
            break
    assert len(picked) == 4
    for t in picked:
        for thr in (t, float(np.nextafter(t, np.inf)), float(np.nextafter(t, -np.inf))):
            su = oracle.setup(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=thr)
            with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=thr) as h:
                assert h.info().n_conflicts == su.info.n_conflicts, thr
                assert np.array_equal(h.groups(), su.group_of), thr


def test_conflicts_with_values_outside_the_filter_range(obk):
    # rows scaled by 2^45 and 2^-45 (and a threshold below 2^-20) leave the
    # range in which FP32 bounds decide the pairs: every pair is then exact
    s = synth.random_dominant(2000, 7, seed=1010)
    A = s.A
    v = A.val.copy()
    for i, scale in ((3, 2.0 ** 45), (700, 2.0 ** -45), (1500, 2.0 ** 45)):
        v[A.row_ptr[i]:A.row_ptr[i + 1]] *= scale
    for thr in (0.1, 2.0 ** -25):
        su = oracle.setup(A.m, A.n, A.row_ptr, A.col_idx, v, s.f, thr=thr)
        with obk.Handle(A.row_ptr, A.col_idx, v, A.m, A.n, thr=thr) as h:
            assert h.info().n_conflicts == su.info.n_conflicts
            assert np.array_equal(h.groups(), su.group_of)


@pytest.mark.parametrize("name", list(CASES))
def test_solve_parity(obk, name):
    s, su = _case(name)
    A = s.A
    tol = 1e-8
    st_o, x_o, io = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=tol, maxit=20000)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        st, x, info = h.solve(s.f, None, tol=tol, maxit=20000)
        assert st == st_o
        assert abs(info.sweeps - io.sweeps) <= 1
        # same number of sweeps, no early stop: x must agree to XTOL
        st2, x2, info2 = h.solve(s.f, None, tol=1e-300, maxit=io.sweeps)
        assert info2.sweeps == io.sweeps
    nrm = np.linalg.norm(x_o)
    err = np.linalg.norm(x2 - x_o) / (nrm if nrm > 0 else 1.0)
    assert err <= XTOL, err
    if info.sweeps == io.sweeps:
        assert np.linalg.norm(x - x_o) / (nrm if nrm > 0 else 1.0) <= XTOL


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_band_waits_equal_grid_barriers(obk, name, precision):
    """The band-local step counters change only when each block runs a step,
    never what a step reads: x must be bit-identical to the solve with a grid
    barrier after every phase, for the same number of sweeps (FP64 and the
    FP32 inner sweeps of the precision form)."""
    s, _ = _case(name)
    A = s.A
    base = dict(precision=precision, inner_sweeps=6) if precision else dict(check_every=1)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        for block in (1024, 512):
            st0, x0, i0 = h.solve(s.f, tol=1e-9, maxit=3000, opts=obk.Opts(sync_mode=2, block_threads=block, **base))
            st1, x1, i1 = h.solve(s.f, tol=1e-9, maxit=3000, opts=obk.Opts(sync_mode=1, block_threads=block, **base))
            assert st0 == st1 and i0.sweeps == i1.sweeps and i0.outer_iters == i1.outer_iters
            assert np.array_equal(x0.view(np.uint64), x1.view(np.uint64)), block


@pytest.mark.parametrize("name", ["knn_30000", "random_dominant_2000"])
def test_adaptive_schedule_parity(obk, name):
    s, _ = _case(name)
    A = s.A
    st_o, x_o, io = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-8, maxit=5000,
                                 check_every=-1)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        st, x, info = h.solve(s.f, None, tol=1e-8, maxit=5000, opts=obk.Opts(check_every=-1))
    assert st == st_o == obk.OBK_OK and info.rel_res <= 1e-8
    assert abs(info.sweeps - io.sweeps) <= 1
    if info.sweeps == io.sweeps:
        assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= XTOL


@pytest.mark.parametrize("rpw", [1, 2, 4, 8, 16, 32])
def test_rows_per_warp_variants_agree(obk, rpw):
    s, su = _case("knn_30000")
    A = s.A
    _, x_o, io = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-300, maxit=4)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        st, x, info = h.solve(s.f, None, tol=1e-300, maxit=4, opts=obk.Opts(rows_per_warp=rpw))
    assert info.sweeps == 4
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= XTOL


def test_autotune_keeps_results_and_parity(obk):
    """The autotuner times every (rows per warp, block size, x/y placement)
    setting; whichever it keeps, and each candidate forced through the options,
    must give the oracle's x after the same sweeps (FP64) and the same result
    as the default setting (precision form)."""
    s, _ = _case("knn_30000")
    A = s.A
    st_o, x_o, io = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-300, maxit=5)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        t = h.autotune(0)
        assert t["rows_per_warp"] in (1, 2, 4, 8, 16, 32) and t["block_threads"] in (512, 1024)
        assert t["staging"] in ("global", "shared") and t["sync"] in ("barriers", "counters") and t["sweep_ms"] > 0
        key = (t["rows_per_warp"], t["block_threads"], t["sync"], t["staging"])
        assert t["candidate_ms"][key] == t["sweep_ms"]
        # a timed candidate reads a positive time (0 = skipped), and the kept one is the fastest
        assert all(ms >= 0 for ms in t["candidate_ms"].values())
        assert t["sweep_ms"] == min(ms for ms in t["candidate_ms"].values() if ms > 0)
        timed = [k for k, ms in t["candidate_ms"].items() if ms > 0]
        assert {(32, b, "counters", p) for b in (1024, 512) for p in ("global", "shared")} <= set(timed)
        assert {(32, b, "barriers", "global") for b in (1024, 512)} <= set(timed)
        t1 = h.autotune(1)
        assert t1["rows_per_warp"] in (1, 2, 4, 8, 16, 32)
        assert all(ms >= 0 for ms in t1["candidate_ms"].values())
        assert t1["sweep_ms"] == min(ms for ms in t1["candidate_ms"].values() if ms > 0)
        st, x, info = h.solve(s.f, None, tol=1e-300, maxit=5)  # the tuned FP64 setting
        assert info.sweeps == 5
        assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= XTOL
        ref32 = {}
        for block in (1024, 512):
            _, ref32[block], _ = h.solve(s.f, None, tol=1e-9, maxit=3000,
                                         opts=obk.Opts(precision=1, rows_per_warp=32, block_threads=block,
                                                       sync_mode=1, staging=2))
        # the residual's partial sums follow the grid, so the two block sizes
        # agree to the parity bound, not bit for bit
        assert np.linalg.norm(ref32[512] - ref32[1024]) <= XTOL * np.linalg.norm(ref32[1024])
        for rpw, block, sync, place in timed:
            knobs = dict(rows_per_warp=rpw, block_threads=block, sync_mode=2 if sync == "counters" else 1,
                         staging=1 if place == "shared" else 2)
            st, x, info = h.solve(s.f, None, tol=1e-300, maxit=5, opts=obk.Opts(**knobs))
            assert info.sweeps == 5
            assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= XTOL, (rpw, block, sync, place)
            if rpw == 32:  # the sliced kernels: ordering and placement change no bit
                _, x32, _ = h.solve(s.f, None, tol=1e-9, maxit=3000, opts=obk.Opts(precision=1, **knobs))
                assert np.array_equal(x32.view(np.uint64), ref32[block].view(np.uint64)), (block, sync, place)


def test_batched_small_systems_match_single_solves(obk):
    import torch

    dev = torch.device("cuda")
    systems = [synth.random_dominant(n, 7, seed=300 + k) for k, n in enumerate((500, 1200, 2000, 3100, 777))]
    systems += [synth.rect_random(2 * n, n, 10, seed=350 + k) for k, n in enumerate((600, 1300))]
    systems += [_zero_rows()]
    handles, fs, outs, ref = [], [], [], []
    for s in systems:
        A = s.A
        h = obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1)
        handles.append(h)
        fs.append(torch.from_numpy(s.f).to(dev))
        outs.append(torch.empty(A.n, dtype=torch.float64, device=dev))
        st_o, x_o, io = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-8, maxit=5000)
        ref.append((st_o, x_o, io))
    sts, infos = obk.solve_batch(handles, fs, outs, tol=1e-8, maxit=5000)
    for (st_o, x_o, io), st, info, out in zip(ref, sts, infos, outs):
        assert st == st_o == obk.OBK_OK
        assert abs(info.sweeps - io.sweeps) <= 1 and info.rel_res <= 1e-8
        if info.sweeps == io.sweeps:
            x = out.cpu().numpy()
            assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= XTOL
    # too large for one block: refused
    big = synth.knn_dominant(30000, 12, seed=5)
    hb = obk.Handle(big.A.row_ptr, big.A.col_idx, big.A.val, big.A.m, big.A.n)
    with pytest.raises(obk.ObkError):
        obk.solve_batch([hb], [torch.from_numpy(big.f).to(dev)], [torch.empty(big.A.n, dtype=torch.float64,
                                                                               device=dev)])
    for h in handles + [hb]:
        h.close()


def test_fixed_sweeps_with_x0_and_device_buffers(obk):
    import torch

    s, su = _case("knn_30000")
    A = s.A
    rng = np.random.default_rng(5)
    x0 = rng.standard_normal(A.n)
    gptr, grows = oracle.group_lists(su.group_of, su.G)
    x0_t = x0[su.perm]
    xt = oracle.sweep(su.N, su.rp, su.ci, su.v, su.nsq, su.f, gptr, grows, x0_t, 3)
    x_o = np.empty_like(xt)
    x_o[su.perm] = xt
    dev = torch.device("cuda")
    with obk.Handle(torch.from_numpy(A.row_ptr).to(dev), torch.from_numpy(A.col_idx).to(dev),
                    torch.from_numpy(A.val).to(dev), A.m, A.n, thr=0.1) as h:
        out = torch.empty(A.n, dtype=torch.float64, device=dev)
        st, _, info = h.solve(torch.from_numpy(s.f).to(dev), torch.from_numpy(x0).to(dev), tol=1e-300,
                              maxit=3, out=out)
        assert st == obk.OBK_NOT_CONVERGED and info.sweeps == 3
        x = out.cpu().numpy()
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= XTOL


def test_deterministic_repeat(obk):
    s, _ = _case("random_dominant_2000")
    A = s.A
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        _, x1, _ = h.solve(s.f, tol=1e-10, maxit=500)
        _, x2, _ = h.solve(s.f, tol=1e-10, maxit=500)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h2:
        _, x3, _ = h2.solve(s.f, tol=1e-10, maxit=500)
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3)


def test_precision_form_reaches_1e10(obk):
    s, _ = _case("knn_30000")
    A = s.A
    st_o, x_o, io = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-10, maxit=20000)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        st, x, info = h.solve(s.f, tol=1e-10, maxit=20000, opts=obk.Opts(precision=1))
    assert st == obk.OBK_OK and info.rel_res <= 1e-10 and info.outer_iters >= 1
    err = np.linalg.norm(x - x_o) / np.linalg.norm(x_o)
    assert err <= 1e-8, err


def test_precision_form_n200k_against_both_oracle_forms(obk):
    """The precision form on the 4M benchmark recipe at n = 200,000 (seed
    1003), to rel. residual 1e-10 with 8 FP32 inner sweeps per refinement step
    on both sides: the GPU result against the FP64 oracle and against the
    oracle's own precision form.  Both sides stop on the same refinement step;
    both results have a residual below 1e-10 on a diagonally dominant system
    (||A^-1|| ||A|| about 5), so they agree with each other and with the FP64
    solve far inside the FP64 parity bound."""
    import torch

    s = synth.knn_dominant(200_000, 12, seed=1003)
    A = s.A
    _, x64, _ = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-10, maxit=20000,
                             check_every=-1)
    st32, x32, i32 = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-10, maxit=20000,
                                  precision=1, inner_sweeps=8)
    assert st32 == oracle.OK
    dev = torch.device("cuda")
    with obk.Handle(torch.from_numpy(A.row_ptr).to(dev), torch.from_numpy(A.col_idx).to(dev),
                    torch.from_numpy(A.val).to(dev), A.m, A.n, thr=0.1) as h:
        out = torch.empty(A.n, dtype=torch.float64, device=dev)
        st, _, info = h.solve(torch.from_numpy(s.f).to(dev), tol=1e-10, maxit=20000, out=out,
                              opts=obk.Opts(precision=1, inner_sweeps=8))
        x = out.cpu().numpy()
    assert st == obk.OBK_OK and info.rel_res <= 1e-10
    assert info.outer_iters == i32.outer_iters and info.sweeps == i32.sweeps
    e64 = np.linalg.norm(x - x64) / np.linalg.norm(x64)
    e32 = np.linalg.norm(x - x32) / np.linalg.norm(x32)
    assert e64 <= XTOL and e32 <= XTOL, (e64, e32)


@pytest.mark.parametrize("name", ["knn_30000", "rect_over_3000x1000"])
def test_select_threshold_probes_match_oracle(obk, name):
    """The residual-feedback threshold choice: for every candidate the groups
    and the residual after the probe sweeps match the oracle's (setup, the same
    number of sweeps from x0 = 0, residual); the choice is the candidate with
    the smallest predicted time; the returned handle is prepared with it."""
    s, _ = _case(name)
    A = s.A
    cands = (0.02, 0.1, 0.3)
    probe = 4
    thr, h, rows = obk.select_threshold(A.row_ptr, A.col_idx, A.val, A.m, A.n, s.f, cands, probe_sweeps=probe,
                                        tol=1e-8)
    try:
        for r in rows:
            su = oracle.setup(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=r["thr"])
            gptr, grows = oracle.group_lists(su.group_of, su.G)
            x = oracle.sweep(su.N, su.rp, su.ci, su.v, su.nsq, su.f, gptr, grows, np.zeros(su.N), nsweeps=probe)
            rr = oracle.residual(su.N, su.rp, su.ci, su.v, su.f, x)
            assert r["groups"] == su.G and r["conflicts"] == su.info.n_conflicts
            assert r["probe_sweeps"] == probe
            assert abs(r["rel_res"] - rr) <= 1e-8 * rr, (r["thr"], r["rel_res"], rr)
            assert abs(r["rate"] - rr ** (1.0 / probe)) <= 1e-8
        best = min(range(len(rows)), key=lambda k: (rows[k]["predicted_ms"], k))
        assert thr == cands[best] and h.G == rows[best]["groups"]
        st, x, info = h.solve(s.f, tol=1e-8, maxit=20000)
        assert st == obk.OBK_OK
    finally:
        h.close()


def test_overdetermined_inconsistent_stagnates(obk):
    s = synth.rect_random(3000, 1000, 10, seed=12, noise=1e-3)
    A = s.A
    st_o, x_o, io = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-8, maxit=5000,
                                 stagnation=1e-12)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        st, x, info = h.solve(s.f, tol=1e-8, maxit=5000, opts=obk.Opts(stagnation=1e-12))
    assert st == st_o == obk.OBK_NOT_CONVERGED
    assert abs(info.sweeps - io.sweeps) <= 10
    assert abs(info.rel_res - io.rel_res) <= 1e-6 * io.rel_res


@pytest.mark.parametrize("name", ["random_dominant_2000", "knn_30000", "rect_over_3000x1000", "zero_rows"])
def test_residual_entry_point(obk, name):
    import torch

    s, _ = _case(name)
    A = s.A
    x = np.random.default_rng(2).standard_normal(A.n)
    rr_host = obk.residual(A.row_ptr, A.col_idx, A.val, A.m, A.n, s.f, x)
    dev = torch.device("cuda")
    rr_dev = obk.residual(torch.from_numpy(A.row_ptr).to(dev), torch.from_numpy(A.col_idx).to(dev),
                          torch.from_numpy(A.val).to(dev), A.m, A.n, torch.from_numpy(s.f).to(dev),
                          torch.from_numpy(x).to(dev))
    assert rr_host == rr_dev  # deterministic: same bits from host or device inputs
    import scipy.sparse as sp

    M = sp.csr_matrix((A.val, A.col_idx, A.row_ptr), shape=(A.m, A.n))
    ref = np.linalg.norm(s.f - M @ x) / np.linalg.norm(s.f)
    assert abs(rr_host - ref) <= 1e-13 * ref


def test_invalid_inputs(obk):
    rp = np.array([0, 2, 3], np.int64)
    ci = np.array([1, 0, 1], np.int32)  # unsorted row 0
    with pytest.raises(obk.ObkError) as e:
        obk.Handle(rp, ci, np.ones(3), 2, 2)
    assert e.value.status == obk.OBK_ERR_INVALID
    with pytest.raises(obk.ObkError) as e:
        obk.Handle(rp, np.array([0, 1, 1], np.int32), np.array([1.0, np.nan, 1.0]), 2, 2)
    assert e.value.status == obk.OBK_ERR_INVALID
    s, _ = _case("tiny_3x3")
    A = s.A
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n) as h:
        with pytest.raises(obk.ObkError):
            h.solve(np.array([1.0, np.inf, 0.0]))
        with pytest.raises(obk.ObkError):
            h.solve(s.f, tol=0.0)


def test_large_pinned_host_matrix(obk):
    # a matrix of more than 2^20 entries in pinned host memory takes the path
    # whose value copy overlaps the reordering (finiteness checked after it):
    # the same setup and solution as from device arrays, and a NaN still
    # rejected as invalid input
    import torch

    s = synth.random_dominant(150000, 7, seed=1011)
    A = s.A
    assert A.nnz >= 1 << 20
    rp_h = torch.from_numpy(A.row_ptr).pin_memory()
    ci_h = torch.from_numpy(A.col_idx).pin_memory()
    v_h = torch.from_numpy(A.val).pin_memory()
    dev = torch.device("cuda:0")
    with obk.Handle(rp_h, ci_h, v_h, A.m, A.n) as hh, \
            obk.Handle(rp_h.to(dev), ci_h.to(dev), v_h.to(dev), A.m, A.n) as hd:
        assert np.array_equal(hh.perm(), hd.perm())
        assert np.array_equal(hh.groups(), hd.groups())
        assert np.array_equal(hh.row_norms().view(np.uint64), hd.row_norms().view(np.uint64))
        _, xh, _ = hh.solve(s.f, tol=1e-8, maxit=2000)
        _, xd, _ = hd.solve(s.f, tol=1e-8, maxit=2000)
        assert np.array_equal(xh, xd)
    v_bad = v_h.clone().pin_memory()
    v_bad[A.nnz // 2] = float("nan")
    with pytest.raises(obk.ObkError) as e:
        obk.Handle(rp_h, ci_h, v_bad, A.m, A.n)
    assert e.value.status == obk.OBK_ERR_INVALID and "non-finite" in str(e.value)


def test_bounded_wait_times_out_and_context_survives(obk):
    # a wait limit of a few polls cannot cover the grid barrier of a multi-block
    # sweep: the kernel must give up, report OBK_ERR_TIMEOUT, and leave the
    # context usable (a one-block grid has no grid barrier, so a larger system)
    s, _ = _case("knn_30000")
    A = s.A
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n) as h:
        with pytest.raises(obk.ObkError) as e:
            h.solve(s.f, tol=1e-8, maxit=50, opts=obk.Opts(timeout_spins=1))
        assert e.value.status == obk.OBK_ERR_TIMEOUT
        st, x, info = h.solve(s.f, tol=1e-8, maxit=5000)
        assert st == obk.OBK_OK


def _serve(obk, srv, reqs, limit_s=300):
    """Submit every (system, opts) of reqs to srv at once; wait for all results."""
    import time

    tickets = []
    for s, o in reqs:
        A = s.A
        tickets.append(srv.submit(A.row_ptr, A.col_idx, A.val, A.m, A.n, s.f, tol=1e-8, maxit=20000, opts=o))
    results = {}
    t0 = time.time()
    while len(results) < len(tickets) and time.time() - t0 < limit_s:
        for t, (s, _) in zip(tickets, reqs):
            if t in results:
                continue
            st, x, info = srv.poll(t, s.A.n)
            if st != obk.OBK_PENDING:
                results[t] = (st, x, info)
        time.sleep(0.005)
    assert len(results) == len(tickets), "requests did not finish"
    return [results[t] for t in tickets]


def test_request_loop_alone_equals_mixed(obk):
    """Each request's result is the same whether it runs alone in the request
    loop or mixed with others that overlap it on the device: small square
    systems (the one-block batch path), overdetermined (Algorithm 5) and
    underdetermined (Algorithm 6) systems, FP64 and FP32 + FP64 refinement
    requests, and kNN systems of 60,000 and 120,000 rows that take the
    cooperative grid path while the small ones run."""
    P64, P32 = obk.Opts(precision=0), obk.Opts(precision=1)
    reqs = []
    for k, n in enumerate((1200, 3000, 800, 5000)):
        reqs.append((synth.random_dominant(n, 7, seed=900 + k), P64 if k % 2 == 0 else P32))
    for k, n in enumerate((700, 1500)):
        reqs.append((synth.rect_random(2 * n, n, 10, seed=950 + k), P32 if k == 0 else P64))
    for k, n in enumerate((4000, 9000)):
        reqs.append((synth.rect_random(n // 2, n, 10, seed=970 + k, full_columns=False), P64 if k == 0 else P32))
    reqs.append((synth.knn_dominant(60_000, 12, seed=980), P32))
    reqs.append((synth.knn_dominant(120_000, 12, seed=981), P64))
    alone = []
    for r in reqs:
        srv = obk.Server(hbm_budget_bytes=0, max_streams=4)
        alone.append(_serve(obk, srv, [r])[0])
        srv.close()
    srv = obk.Server(hbm_budget_bytes=0, max_streams=4)
    mixed = _serve(obk, srv, reqs)
    srv.close()
    for k, ((st_a, x_a, i_a), (st_m, x_m, i_m)) in enumerate(zip(alone, mixed)):
        assert st_a == st_m == obk.OBK_OK, (k, st_a, st_m)
        assert i_m.sweeps == i_a.sweeps, (k, i_a.sweeps, i_m.sweeps)
        assert np.linalg.norm(x_m - x_a) <= XTOL * np.linalg.norm(x_a), k


def _wait(srv, ticket, n, limit_s=120):
    import time

    t0 = time.time()
    while time.time() - t0 < limit_s:
        st, x, info = srv.poll(ticket, n)
        if st != obk_pending():
            return st, x, info
        time.sleep(0.005)
    raise AssertionError("request did not finish")


def obk_pending():
    import paper_2401_00672_gb300 as m

    return m.OBK_PENDING


def test_request_loop_budget_cancel_and_unknown_ticket(obk):
    s, _ = _case("knn_30000")
    A = s.A
    # a request that can never fit the budget is refused at submission
    tiny = obk.Server(hbm_budget_bytes=1 << 20, max_streams=1)
    with pytest.raises(obk.ObkError) as e:
        tiny.submit(A.row_ptr, A.col_idx, A.val, A.m, A.n, s.f)
    assert e.value.status == obk.OBK_ERR_BUDGET
    tiny.close()
    # one worker: the second request waits in the queue and can be cancelled there
    srv = obk.Server(hbm_budget_bytes=0, max_streams=1)
    t1 = srv.submit(A.row_ptr, A.col_idx, A.val, A.m, A.n, s.f, tol=1e-8, maxit=5000)
    t2 = srv.submit(A.row_ptr, A.col_idx, A.val, A.m, A.n, s.f, tol=1e-8, maxit=5000)
    assert srv.cancel(t2) == obk.OBK_OK
    st1, x1, _ = _wait(srv, t1, A.n)
    st2, _, _ = _wait(srv, t2, A.n)
    assert st1 == obk.OBK_OK and st2 == obk.OBK_ERR_CANCELLED
    # a finished ticket is released by its final poll
    st, _, _ = srv.poll(t1, A.n)
    assert st == obk.OBK_ERR_NOT_FOUND
    assert srv.cancel(123456789) == obk.OBK_ERR_NOT_FOUND
    srv.close()
    _, x_alone, _ = obk.solve(A.row_ptr, A.col_idx, A.val, A.m, A.n, s.f, tol=1e-8, maxit=5000)
    assert np.linalg.norm(x1 - x_alone) <= XTOL * np.linalg.norm(x_alone)


def test_request_loop_budget_admits_one_at_a_time(obk):
    # the budget fits one request at a time: all still finish, in arrival order
    systems = [synth.random_dominant(3000 + 500 * k, 7, seed=700 + k) for k in range(4)]
    foot = max(obk.request_footprint(s.A.m, s.A.n, s.A.nnz) for s in systems)
    srv = obk.Server(hbm_budget_bytes=foot + 1024, max_streams=4)
    tickets = [srv.submit(s.A.row_ptr, s.A.col_idx, s.A.val, s.A.m, s.A.n, s.f, tol=1e-8, maxit=5000)
               for s in systems]
    for t, s in zip(tickets, systems):
        st, x, info = _wait(srv, t, s.A.n)
        assert st == obk.OBK_OK and info.rel_res <= 1e-8
    srv.close()


@pytest.mark.slow
def test_full_size_knn_1m_parity(obk):
    """The kNN workload at n = 1,000,000, in the configuration the benchmark
    times: setup bit-exact and x within 1e-9 at the oracle's stopping sweep."""
    s = synth.knn_dominant(1_000_000, 12, seed=1001)
    A = s.A
    st_o, x_o, io, perm_o, gof_o = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-8,
                                                maxit=10000, return_setup=True)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        assert np.array_equal(h.perm(), perm_o)
        assert np.array_equal(h.groups(), gof_o)
        st, x, info = h.solve(s.f, tol=1e-8, maxit=10000)
        assert st == st_o == obk.OBK_OK and abs(info.sweeps - io.sweeps) <= 1
        st2, x2, _ = h.solve(s.f, tol=1e-300, maxit=io.sweeps)
    assert np.linalg.norm(x2 - x_o) / np.linalg.norm(x_o) <= XTOL


def test_knn_2m_two_column_mirror_slices(obk):
    # at n = 2,000,000 the largest groups' (group, tile) pieces hold more than
    # 4096 column segments, so their mirror slices carry two columns per lane
    # (the smaller groups' one): setup bit-exact, the FP64 x after a fixed
    # number of sweeps and the FP32 + refinement x within 1e-9 of the oracle
    s = synth.knn_dominant(2_000_000, 12, seed=1012)
    A = s.A
    k = 6
    st_o, x_o, io, perm_o, gof_o = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-300,
                                                maxit=k, return_setup=True)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        assert np.array_equal(h.perm(), perm_o)
        assert np.array_equal(h.groups(), gof_o)
        for sync in (1, 2):
            _, x, info = h.solve(s.f, tol=1e-300, maxit=k, opts=obk.Opts(sync_mode=sync))
            assert info.sweeps == k
            assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= XTOL
        st, x32, info = h.solve(s.f, tol=1e-10, maxit=20000, opts=obk.Opts(precision=1))
        assert st == obk.OBK_OK and info.rel_res <= 1e-10
    st64, x64, _ = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-10, maxit=20000)
    assert st64 == oracle.OK
    assert np.linalg.norm(x32 - x64) / np.linalg.norm(x64) <= XTOL


@pytest.mark.parametrize("name", list(CASES))
def test_cosine_stats_bit_exact(obk, name):
    """Definitions 1-2 from the GPU equal the oracle's on the permuted matrix."""
    s, su = _case(name)
    A = s.A
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        g = h.grouping_stats()
    N = su.N
    # the oracle's extended (Algorithms 5/6: N = max(m, n), appended rows empty)
    # and permuted matrix
    rp_ext = np.concatenate([A.row_ptr, np.full(N - A.m, A.row_ptr[-1], np.int64)])
    rp, ci, v = oracle.permute(N, rp_ext, A.col_idx, A.val, su.perm)
    nsq = oracle.row_norms(N, rp, v)
    nz, tot, zn, nn = oracle.cosine_stats(N, rp, ci, v, nsq)
    assert g["N"] == N
    assert g["nonzero_entries"] == nz and g["abs_cos_sum"] == tot
    assert g["zn"] == pytest.approx(zn, rel=1e-15) and g["nn"] == pytest.approx(nn, rel=1e-15)
    assert g["groups"] == su.G
    # conflicting pairs as the oracle's grouping counts them; the fixed point
    # needs at least one round (and a last one that changes nothing)
    _, _, n_conf = oracle.group_build(N, rp, ci, v, nsq, 0.1)
    assert g["conflicts"] == n_conf
    assert g["color_rounds"] >= (2 if n_conf else 1)


def test_underdetermined_min_norm(obk):
    """UOBK (Algorithm 6) from x0 = 0 ends at the minimum-norm solution of a
    consistent underdetermined system (full row rank): compare with numpy's
    least-squares minimum-norm solution."""
    s = synth.rect_random(300, 800, 8, seed=11, full_columns=False)
    A = s.A
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        st, x, info = h.solve(s.f, None, tol=1e-12, maxit=200000)
    assert st == 0
    xmn = np.linalg.lstsq(A.to_dense(), s.f, rcond=None)[0]
    assert np.linalg.norm(x - xmn) / np.linalg.norm(xmn) < 1e-9


@pytest.mark.parametrize("name", ["random_dominant_2000", "knn_30000", "rect_over_3000x1000", "hubs"])
def test_pinv_group_steps_parity(obk, name):
    """Eq. 1.3 group steps (K Jacobi steps on each group's Gram system) against
    the oracle with the same K."""
    s, su = _case(name)
    A = s.A
    K = 8
    st_o, x_o, io = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-8, maxit=20000,
                                 pinv_iters=K)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        st, x, info = h.solve(s.f, None, tol=1e-8, maxit=20000, opts=obk.Opts(pinv_iters=K))
        st0, x0, info0 = h.solve(s.f, None, tol=1e-8, maxit=20000)  # the default step afterwards
    assert st == st_o == 0
    assert abs(info.sweeps - io.sweeps) <= 1
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= XTOL
    assert st0 == 0


def test_pinv_iters_rejected_where_unsupported(obk):
    s, _ = _case("tiny_3x3")
    A = s.A
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        with pytest.raises(obk.ObkError):
            h.solve(s.f, None, opts=obk.Opts(pinv_iters=-1))


@pytest.mark.parametrize("name,k", [("random_dominant_2000", 8), ("knn_30000", 6), ("rect_over_3000x1000", 5),
                                    ("rect_under_400x1000", 4), ("components", 3), ("diag", 7)])
def test_block_form_parity(obk, name, k):
    """Algorithm 4 as printed (k uniform blocks, centroid-cosine classes, CGLS
    projections): the same classes as the oracle, and x within 1e-8.

    The bound is looser than the row-group form's 1e-9 because each block
    projection is itself an iteration: both sides stop their CGLS runs when the
    normal-equation residual fell below 1e-13 of its start, and the two runs
    (different summation orders of the same FP64 arithmetic) can stop a step
    apart, so each projection is reproduced only to that inner tolerance times
    the block's conditioning; over ~10 iterations of the outer loop, a few 1e-9
    of x separate the two results, not rounding."""
    s, _ = _case(name)
    A = s.A
    tol = 1e-9
    st_o, x_o, io, np_o, nq_o = oracle.solve_blocks(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, k=k, thr=0.1,
                                                    tol=tol, maxit=3000)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        st, x, info, bo = h.solve_blocks(s.f, None, k=k, thr=0.1, tol=tol, maxit=3000)
    assert (bo.n_pairs, bo.n_nclass) == (np_o, nq_o)
    assert st == st_o == 0
    assert abs(info.sweeps - io.sweeps) <= 1
    assert np.linalg.norm(x - x_o) / max(np.linalg.norm(x_o), 1e-300) <= 1e-8


def _dense_conflicts(N=2000, hubs=6, per_row=4, seed=61):
    # every row has entries in per_row of a few shared columns: each row
    # conflicts with hundreds of earlier rows (whole-warp conflict lists and
    # more than 64 groups)
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(N):
        c = rng.choice(np.arange(N - hubs, N), per_row, replace=False)
        c = c[c != i]
        rows += [i] * len(c)
        cols += list(c)
    r = np.array(rows, np.int64)
    c = np.array(cols, np.int64)
    v = rng.standard_normal(len(r))
    off = np.bincount(r, weights=np.abs(v), minlength=N)
    r = np.concatenate([r, np.arange(N)])
    c = np.concatenate([c, np.arange(N)])
    v = np.concatenate([v, 1.0 + off])
    A = synth.csr_from_coo(N, N, r, c, v)
    xs = rng.standard_normal(N)
    return synth.System(A, xs, A.matvec(xs), "dense_conflicts")


def test_dense_conflicts_wide_lanes(obk):
    """Conflict lists of hundreds of rows (the grouping's whole-warp path, more
    than 64 colours): setup bit-exact and a fixed number of sweeps in parity."""
    s = _dense_conflicts()
    A = s.A
    su = oracle.setup(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1)
    with obk.Handle(A.row_ptr, A.col_idx, A.val, A.m, A.n, thr=0.1) as h:
        g = h.grouping_stats()
        assert g["conflicts"] > 96 * su.N  # more than 96 per row: 32 lanes per row
        assert h.G == su.G and su.G > 64
        assert np.array_equal(h.perm(), su.perm)
        assert np.array_equal(h.groups(), su.group_of)
        assert h.info().n_conflicts == su.info.n_conflicts
        st, x, info = h.solve(s.f, tol=1e-300, maxit=5)
    st_o, x_o, io = oracle.solve(A.m, A.n, A.row_ptr, A.col_idx, A.val, s.f, thr=0.1, tol=1e-300, maxit=5)
    assert info.sweeps == io.sweeps == 5
    assert np.linalg.norm(x - x_o) / np.linalg.norm(x_o) <= XTOL
