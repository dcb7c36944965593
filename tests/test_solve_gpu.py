"""Parity of lu_solve (and the batched entry points) with the oracle."""
import numpy as np
import pytest

import lu_inputs as li
from tests._parity import EPS32, oracle_parity
from tests.gpu_util import EPS64, dev, factor_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,nrhs", [(1, 1), (65, 3), (512, 1), (700, 17)])
def test_solve_f64_matches_oracle(oracle_mod, n, nrhs):
    import torch

    import paper_1611_06365_gb300 as lu
    A = li.uniform(n, n, seed=30 + n)
    B = li.uniform(n, nrhs, seed=31 + n)
    LU, ipiv, info, dA, dpiv = factor_gpu(A, "f64")
    dB = li.to_device_colmajor(B, dev())
    lu.lu_solve(dA, dpiv, dB, n)
    torch.cuda.synchronize()
    X = li.from_device_colmajor(dB, n)
    LUo, pivo, _ = oracle_mod.getrf(A)
    Xo = oracle_mod.getrs(LUo, pivo, B)
    assert np.max(np.abs(X - Xo)) <= 1e3 * n * EPS64 * max(1.0, np.max(np.abs(Xo)))
    assert oracle_mod.backward_error(A, X, B) <= 10 * n * EPS64


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_solve_rhs_independent_bits(dtype):
    """The right-hand sides of a pass run as separate substitution chains (one or
    two per chain): every column of a multi-column solve equals the solve of
    that column alone, bit for bit, for 1..8 columns (chains of one), 9..16
    (chains of two, a ragged last chain) and beyond 16 (several passes)."""
    import torch

    import paper_1611_06365_gb300 as lu
    n = 777
    A = li.uniform(n, n, seed=41)
    B = li.uniform(n, 35, seed=42)
    _, _, _, dA, dpiv = factor_gpu(A, dtype)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    single = []
    for q in range(B.shape[1]):
        dB = li.to_device_colmajor(B[:, q:q + 1], dev(), dtype=tdt)
        lu.lu_solve(dA, dpiv, dB, n)
        single.append(li.from_device_colmajor(dB, n)[:, 0])
    torch.cuda.synchronize()
    for nrhs in (2, 8, 11, 16, 35):
        dB = li.to_device_colmajor(B[:, :nrhs], dev(), dtype=tdt)
        lu.lu_solve(dA, dpiv, dB, n)
        torch.cuda.synchronize()
        X = li.from_device_colmajor(dB, n)
        for q in range(nrhs):
            assert np.array_equal(X[:, q], single[q]), (nrhs, q)


def test_solve_dyadic_exact():
    import torch

    import paper_1611_06365_gb300 as lu
    n = 300
    A, perm, L, U = li.dyadic_plu(n, seed=3)
    x = ((li.splitmix64(6, np.arange(n, dtype=np.uint64)) % np.uint64(9)).astype(np.int64) - 4).astype(float)
    b = A @ x
    LU, ipiv, info, dA, dpiv = factor_gpu(A, "f64")
    dB = torch.from_numpy(b).to(dev()).view(1, n).clone()
    lu.lu_solve(dA, dpiv, dB, n)
    torch.cuda.synchronize()
    assert np.array_equal(dB.view(-1).cpu().numpy(), x)


def test_c1_factor_and_solve_ones(oracle_mod):
    """n = 512 workload: b = A * ones; the solution is ones to rounding."""
    import torch

    import paper_1611_06365_gb300 as lu
    A = li.uniform(512, 512, seed=li.BASE_SEED + 1000)
    b = li.ones_rhs(A)
    LU, ipiv, info, dA, dpiv = factor_gpu(A, "f64")
    dB = torch.from_numpy(b).to(dev()).view(1, 512).clone()
    lu.lu_solve(dA, dpiv, dB, 512)
    torch.cuda.synchronize()
    x = dB.view(-1).cpu().numpy()
    xo = oracle_mod.getrs(*oracle_mod.getrf(A)[:2], b)
    assert np.max(np.abs(x - xo)) < 1e-11
    assert oracle_mod.backward_error(A, x, b) <= 10 * 512 * EPS64


def _batch_buffers(mats, dtype):
    import torch
    tdt = torch.float64 if dtype == "f64" else torch.float32
    devA = [li.to_device_colmajor(a, dev(), dtype=tdt) for a in mats]
    piv = [torch.zeros(max(1, a.shape[0]), dtype=torch.int32, device=dev()) for a in mats]
    ns = torch.tensor([a.shape[0] for a in mats], dtype=torch.int32, device=dev())
    ptrA = torch.tensor([t.data_ptr() for t in devA], dtype=torch.int64, device=dev())
    ptrP = torch.tensor([t.data_ptr() for t in piv], dtype=torch.int64, device=dev())
    lds = ns.clone().clamp(min=1)
    info = torch.zeros(len(mats), dtype=torch.int32, device=dev())
    return devA, piv, ns, ptrA, ptrP, lds, info


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_matches_oracle(oracle_mod, dtype):
    import torch

    import paper_1611_06365_gb300 as lu
    sizes = li.batch_sizes(60, 16, 256, seed=li.BASE_SEED + 3000)
    sizes[:3] = [256, 16, 1]
    mats = li.batch_matrices(sizes, seed=li.BASE_SEED + 3001)
    rhs = [li.ones_rhs(a) for a in mats]
    devA, piv, ns, ptrA, ptrP, lds, info = _batch_buffers(mats, dtype)
    code = lu.LU_F64 if dtype == "f64" else lu.LU_F32
    lu.lu_factor_batched(code, ns, ptrA, lds, ptrP, info, 256)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    devB = [torch.from_numpy(b).to(dev(), tdt).view(1, -1).clone() for b in rhs]
    ptrB = torch.tensor([t.data_ptr() for t in devB], dtype=torch.int64, device=dev())
    lu.lu_solve_batched(code, 1, ns, ptrA, lds, ptrP, ptrB, lds, 256)
    torch.cuda.synchronize()
    LUs, pivs, infos, xs = oracle_mod.getrf_getrs_batched(mats, rhs)
    assert np.array_equal(info.cpu().numpy(), infos)
    for t, A in enumerate(mats):
        n = A.shape[0]
        gp = piv[t].cpu().numpy()[:n]
        if t % 2 == 1:
            assert np.array_equal(gp, np.arange(1, n + 1))
        if dtype == "f64":
            assert np.array_equal(gp, pivs[t]), t
            LU = li.from_device_colmajor(devA[t], n)
            assert np.max(np.abs(LU - LUs[t])) <= 10 * n * EPS64 * max(1.0, np.max(np.abs(LUs[t])))
            assert np.max(np.abs(devB[t].view(-1).cpu().numpy() - xs[t])) <= 1e-9
        else:
            # the whole pivot vector against the oracle run on the FP32-rounded matrix (near
            # ties at FP32 resolution re-run with the GPU's choice), then the factors
            A32 = A.astype(np.float32).astype(np.float64)
            LU = li.from_device_colmajor(devA[t], n)
            LUo32, _ = oracle_parity(oracle_mod, A32, gp, max_reruns=64, threads=1, eps=EPS32)
            assert np.max(np.abs(LU - LUo32)) <= 64 * n * EPS32 * max(1.0, float(np.max(np.abs(LUo32)))), t
            r, a = oracle_mod.lu_residual_fro(A32, LU, gp)
            assert r / a <= 10 * n * 1.2e-7
            assert np.max(np.abs(devB[t].view(-1).cpu().numpy() - 1.0)) <= 1e-2


def test_batched_dyadic_exact():
    import paper_1611_06365_gb300 as lu
    import torch
    mats, perms = [], []
    for i, n in enumerate([16, 33, 100, 256, 200]):
        A, perm, L, U = li.dyadic_plu(n, seed=70 + i)
        mats.append(A)
        perms.append((perm, L, U))
    devA, piv, ns, ptrA, ptrP, lds, info = _batch_buffers(mats, "f64")
    lu.lu_factor_batched(lu.LU_F64, ns, ptrA, lds, ptrP, info, 256)
    torch.cuda.synchronize()
    from tests.gpu_util import expected_ipiv
    for t, (perm, L, U) in enumerate(perms):
        n = L.shape[0]
        LU = li.from_device_colmajor(devA[t], n)
        assert np.array_equal(piv[t].cpu().numpy()[:n], expected_ipiv(perm))
        assert np.array_equal(np.triu(LU), U) and np.array_equal(np.tril(LU, -1) + np.eye(n), L)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_blocked_equals_unblocked(dtype):
    """The blocked batched kernel (panel widths 16 and 32) applies every element's
    fused multiply-adds in the unblocked order: factors, pivots and info are the
    same bits as the unblocked kernel's (nb = 1), ragged orders, a singular member
    and a member with ties included."""
    import torch

    import paper_1611_06365_gb300 as lu
    sizes = [1, 2, 15, 16, 17, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256]
    mats = li.batch_matrices(np.array(sizes), seed=li.BASE_SEED + 3100)
    mats.append(np.zeros((40, 40)))                     # every pivot zero
    sing = li.uniform(70, 70, seed=3101)
    sing[:, 35] = 0.0                                   # zero column: info = 36 unless an earlier pivot is zero
    mats.append(sing)
    mats.append(li.wilkinson(48))                       # magnitude ties in every column
    code = lu.LU_F64 if dtype == "f64" else lu.LU_F32
    results = {}
    for nb in (1, 16, 32):
        devA, piv, ns, ptrA, ptrP, lds, info = _batch_buffers(mats, dtype)
        lu.lu_factor_batched(code, ns, ptrA, lds, ptrP, info, 256, nb=nb)
        torch.cuda.synchronize()
        results[nb] = ([t.cpu().numpy().copy() for t in devA], [p.cpu().numpy().copy() for p in piv], info.cpu().numpy().copy())
    ref = results[1]
    assert ref[2][-3] == 1 and ref[2][-2] > 0
    for nb in (16, 32):
        got = results[nb]
        assert np.array_equal(got[2], ref[2])
        for t in range(len(mats)):
            assert np.array_equal(got[1][t], ref[1][t]), (nb, t)
            assert np.array_equal(got[0][t].view(np.uint8), ref[0][t].view(np.uint8)), (nb, t)
