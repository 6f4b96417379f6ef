"""obk_residual_noalloc against obk_residual.

The allocation-free entry point serves callers that cannot allocate device
memory when they need a residual (memory held by another allocator, or a loop
that cannot afford an allocation).  It must give the same relative residual as
the allocating entry point, on two calls in a row (the second call reuses the
fixed scratch the first one left behind).  This file is collected last, and
passes both alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-13  # same bound as the residual entry-point test


def test_noalloc_residual_matches_allocating_entry_point_twice():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_00672_gb300 as obk

    dev = torch.device("cuda")
    cases = [synth.knn_dominant(20000, 12, seed=31), synth.rect_random(9000, 3000, 10, seed=32)]
    for s in cases:
        A = s.A
        rng = np.random.default_rng(7)
        for call in range(2):
            x = rng.standard_normal(A.n)
            ref = obk.residual(A.row_ptr, A.col_idx, A.val, A.m, A.n, s.f, x)
            out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            obk.residual_noalloc(torch.from_numpy(A.row_ptr).to(dev), torch.from_numpy(A.col_idx).to(dev),
                                 torch.from_numpy(A.val).to(dev), A.m, A.n, torch.from_numpy(s.f).to(dev),
                                 torch.from_numpy(x).to(dev), out)
            torch.cuda.synchronize()
            got = float(out.item())
            assert abs(got - ref) <= RTOL * ref, (call, got, ref)


def test_noalloc_rejects_oversize_and_host_arrays():
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
