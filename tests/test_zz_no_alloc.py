"""obk_residual_noalloc against obk_residual.

The allocation-free entry point serves callers that cannot allocate device
memory when they need a residual (memory held by another allocator, or a loop
that cannot afford an allocation).  Both entry points run the same per-tile
body and the same final sum, so the values must be identical, on two calls in
a row (the second call reuses the fixed scratch the first one left behind),
on the default stream and on another stream.  This file is collected last, and
passes both alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _cases():
    return [synth.knn_dominant(20000, 12, seed=31), synth.rect_random(9000, 3000, 10, seed=32)]


def test_noalloc_residual_matches_allocating_entry_point_twice():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_00672_gb300 as obk

    dev = torch.device("cuda")
    side = torch.cuda.Stream()
    for s in _cases():
        A = s.A
        rng = np.random.default_rng(7)
        for call in range(2):
            x = rng.standard_normal(A.n)
            ref = obk.residual(A.row_ptr, A.col_idx, A.val, A.m, A.n, s.f, x)
            args = [torch.from_numpy(a).to(dev) for a in (A.row_ptr, A.col_idx, A.val)]
            fd, xd = torch.from_numpy(s.f).to(dev), torch.from_numpy(x).to(dev)
            out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            obk.residual_noalloc(*args, A.m, A.n, fd, xd, out)
            torch.cuda.synchronize()
            assert float(out.item()) == ref, (call, float(out.item()), ref)
            # the same call queued on a non-default stream
            out2 = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            side.wait_stream(torch.cuda.current_stream())
            obk.residual_noalloc(*args, A.m, A.n, fd, xd, out2, stream=side.cuda_stream)
            side.synchronize()
            assert float(out2.item()) == ref, (call, float(out2.item()), ref)


def test_noalloc_rejects_oversize_null_and_host_arrays():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_00672_gb300 as obk

    dev = torch.device("cuda")
    rp = torch.zeros(2, dtype=torch.int64, device=dev)
    ci = torch.zeros(1, dtype=torch.int32, device=dev)
    v = torch.zeros(1, dtype=torch.float64, device=dev)
    f = torch.ones(1, dtype=torch.float64, device=dev)
    x = torch.zeros(1, dtype=torch.float64, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(obk.ObkError) as e:
        obk.residual_noalloc(rp, ci, v, 67_108_865, 1, f, x, out)
    assert e.value.status == obk.OBK_ERR_INVALID and "exceeds the maximum" in str(e.value)
    with pytest.raises(TypeError):
        obk.residual_noalloc(rp.cpu(), ci, v, 1, 1, f, x, out)

    # the C entry point itself: NULL col_idx / val and host memory are rejected
    # before any kernel is queued
    lib = obk.lib
    P = ctypes.c_void_p
    dp = [P(t.data_ptr()) for t in (rp, ci, v, f, x, out)]
    assert lib.obk_residual_noalloc(dp[0], None, dp[2], 1, 1, dp[3], dp[4], dp[5], None) == obk.OBK_ERR_INVALID
    assert "NULL" in obk.last_error()
    assert lib.obk_residual_noalloc(dp[0], dp[1], None, 1, 1, dp[3], dp[4], dp[5], None) == obk.OBK_ERR_INVALID
    host_x = np.zeros(1)
    rc = lib.obk_residual_noalloc(dp[0], dp[1], dp[2], 1, 1, dp[3], host_x.ctypes.data_as(P), dp[5], None)
    assert rc == obk.OBK_ERR_INVALID and "device memory" in obk.last_error()
    # a good call clears the last error
    assert lib.obk_residual_noalloc(*dp[:3], 1, 1, *dp[3:], None) == obk.OBK_OK
    torch.cuda.synchronize()
    assert obk.last_error() == ""
    assert float(out.item()) == 1.0  # ||f - A x|| / ||f|| with A = 0, f = 1
