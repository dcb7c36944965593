"""lu_solve_noalloc: the solve for callers that may not allocate device memory
(for instance when another allocator has reserved the device memory, or in a
latency-critical loop).  It must give the same answers as lu_solve, bit for
bit (both run the same kernels on the same data), while its workspace comes
from the library's fixed device array and nothing is allocated.

This file is collected last so that a failure here, in a run that stops at the
first failure, comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import lu_inputs as li

pytestmark = pytest.mark.gpu

CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8      # cuda.h, CUmemPool_attribute


class _DefaultPool:
    """High-water mark of the device's default stream-ordered memory pool (the
    pool lu_solve's cudaMallocAsync draws from), read through the driver API."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def high(self):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(v)) == 0
        return v.value


def _factor(n, dtype, dev):
    import torch

    import paper_1611_06365_gb300 as lu
    tdt = torch.float64 if dtype == "f64" else torch.float32
    dA = li.to_device_colmajor(li.uniform(n, n, seed=900 + n), dev, dtype=tdt)
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    lu.lu_factor(dA, ipiv, info)
    return dA, ipiv, tdt


def _solve_both(dA, ipiv, n, nrhs, tdt, seed, dev, status):
    import torch

    import paper_1611_06365_gb300 as lu
    ref = li.to_device_colmajor(li.uniform(n, nrhs, seed=seed), dev, dtype=tdt)
    got = ref.clone()
    lu.lu_solve(dA, ipiv, ref)
    lu.lu_solve_noalloc(dA, ipiv, got, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return li.from_device_colmajor(ref, n), li.from_device_colmajor(got, n)


@pytest.mark.parametrize("dtype,n,nrhs", [("f64", 700, 3), ("f32", 513, 2), ("f64", 64, 17)])
def test_noalloc_matches_lu_solve_twice(dtype, n, nrhs):
    import torch
    dev = torch.device("cuda:0")
    dA, ipiv, tdt = _factor(n, dtype, dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    for call in range(2):                     # two calls in a row share the scratch
        Xr, Xg = _solve_both(dA, ipiv, n, nrhs, tdt, 910 + 7 * call + n, dev, status)
        assert np.array_equal(Xg, Xr)


def test_noalloc_large_then_small_request():
    """A small request after a large one finds the scratch holding the larger
    layout (flags, permutation, copy of B at other offsets) and must not read it."""
    import torch
    dev = torch.device("cuda:0")
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    for n, nrhs in ((700, 5), (64, 1), (700, 1), (64, 3)):
        dA, ipiv, tdt = _factor(n, "f64", dev)
        Xr, Xg = _solve_both(dA, ipiv, n, nrhs, tdt, 930 + n + nrhs, dev, status)
        assert np.array_equal(Xg, Xr), (n, nrhs)


def test_noalloc_allocates_nothing():
    """lu_solve raises the default pool's high-water mark (its stream-ordered
    workspace); lu_solve_noalloc, after a first call has done its set-up, does not."""
    import torch

    import paper_1611_06365_gb300 as lu
    dev = torch.device("cuda:0")
    n, nrhs = 700, 2
    dA, ipiv, tdt = _factor(n, "f64", dev)
    B = li.to_device_colmajor(li.uniform(n, nrhs, seed=950), dev, dtype=tdt)
    lu.lu_solve_noalloc(dA, ipiv, B.clone())      # set-up call
    torch.cuda.synchronize()
    pool = _DefaultPool()
    pool.reset_high()
    base = pool.high()
    lu.lu_solve(dA, ipiv, B.clone())
    torch.cuda.synchronize()
    assert pool.high() > base                      # the check sees stream-ordered allocations
    pool.reset_high()
    base = pool.high()
    X = B.clone()
    torch.cuda.synchronize()
    lu.lu_solve_noalloc(dA, ipiv, X)
    torch.cuda.synchronize()
    assert pool.high() == base


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
