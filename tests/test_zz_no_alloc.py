"""lu_solve_noalloc: the solve for callers that may not allocate device memory
(for instance when another allocator has reserved the device memory, or in a
latency-critical loop).  It must give the same answers as lu_solve while its
workspace comes from the library's fixed device array.

This file is collected last so that a failure here, in a run that stops at the
first failure, comes after every other test has run.
"""
import numpy as np
import pytest

import lu_inputs as li

pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps
EPS32 = float(np.finfo(np.float32).eps)


@pytest.mark.parametrize("dtype,n,nrhs", [("f64", 700, 3), ("f32", 513, 2), ("f64", 64, 17)])
def test_noalloc_matches_lu_solve_twice(dtype, n, nrhs):
    import torch

    import paper_1611_06365_gb300 as lu
    dev = torch.device("cuda:0")
    tdt = torch.float64 if dtype == "f64" else torch.float32
    eps = EPS64 if dtype == "f64" else EPS32
    A = li.uniform(n, n, seed=900 + n)
    dA = li.to_device_colmajor(A, dev, dtype=tdt)
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    lu.lu_factor(dA, ipiv, info)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    for call in range(2):                     # two calls in a row share the scratch
        B = li.uniform(n, nrhs, seed=910 + 7 * call + n)
        ref = li.to_device_colmajor(B, dev, dtype=tdt)
        got = ref.clone()
        lu.lu_solve(dA, ipiv, ref)
        lu.lu_solve_noalloc(dA, ipiv, got, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        Xr, Xg = li.from_device_colmajor(ref, n), li.from_device_colmajor(got, n)
        assert np.max(np.abs(Xg - Xr)) <= 1e3 * n * eps * max(1.0, np.max(np.abs(Xr)))


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch

    import paper_1611_06365_gb300 as lu
    cap = lu.lu_solve_noalloc_capacity()
    assert cap == 4 << 20
    n, nrhs = 4096, cap // (8 * 4096) + 1      # n * nrhs doubles alone exceed the array
    dev = torch.device("cuda:0")
    LU = torch.zeros((1, 1), dtype=torch.float64, device=dev)
    ipiv = torch.zeros(1, dtype=torch.int32, device=dev)
    B = torch.zeros((1, 1), dtype=torch.float64, device=dev)
    rc = lu.lib().lu_solve_noalloc(lu.LU_F64, n, nrhs, LU.data_ptr(), n, ipiv.data_ptr(), B.data_ptr(), n, None, None)
    assert rc == lu.LU_ERR_SCRATCH
    assert "scratch" in lu.lu_status_string(rc)
