"""Mixed-precision solve (FP32 factors with a BF16 tensor-core update, FP64
refinement) and the BF16 trailing-update kernel on its own."""
import numpy as np
import pytest

import lu_inputs as li
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu


def _bf16(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).float().bfloat16().double().numpy()


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (300, 200, 256), (1000, 77, 100), (5, 3, 16), (700, 900, 192)])
def test_trailing_update_bf16_vs_fp32_reference(m, n, k, split):
    """C - A B with A, B rounded to BF16 (split: x = hi + lo, products
    hi*hi + hi*lo + lo*hi): every product of two BF16 values is exact in
    FP32, so the only difference from an exact sum of the same products is
    FP32 accumulation: |err| <= k' eps32 sum |a||b| + eps32 |C - AB|,
    k' the number of products summed."""
    import torch

    import paper_1611_06365_gb300 as lu
    A = li.uniform(m, k, seed=1 + m)
    B = li.uniform(k, n, seed=2 + n)
    C = li.uniform(m, n, seed=3 + k)
    dA = li.to_device_colmajor(A, dev(), torch.float32)
    dB = li.to_device_colmajor(B, dev(), torch.float32)
    dC = li.to_device_colmajor(C, dev(), torch.float32)
    mode = lu.LU_UPDATE_BF16X3 if split else lu.LU_UPDATE_BF16
    lu.lu_trailing_update(mode, dA, dB, dC, m, n, k)
    torch.cuda.synchronize()
    got = li.from_device_colmajor(dC, m)
    A32 = A.astype(np.float32).astype(np.float64)
    B32 = B.astype(np.float32).astype(np.float64)
    C32 = C.astype(np.float32).astype(np.float64)
    Ah, Bh = _bf16(A32), _bf16(B32)
    if split:
        Al = _bf16((A32 - Ah).astype(np.float32).astype(np.float64))
        Bl = _bf16((B32 - Bh).astype(np.float32).astype(np.float64))
        prod = Ah @ Bh + Ah @ Bl + Al @ Bh
        mag = np.abs(Ah) @ np.abs(Bh) + np.abs(Ah) @ np.abs(Bl) + np.abs(Al) @ np.abs(Bh)
        kk = 3 * k
        # the split really is more accurate than one BF16 product
        assert np.max(np.abs(prod - A32 @ B32)) < 2.0 ** -14 * np.max(np.abs(A32) @ np.abs(B32))
    else:
        prod, mag, kk = Ah @ Bh, np.abs(Ah) @ np.abs(Bh), k
    ref = C32 - prod
    bound = kk * 2.0 ** -23 * mag + 2.0 ** -23 * np.abs(ref) + 1e-30
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)


def _e4m3(x):
    """Round to nearest (ties to even) onto the e4m3 grid: 3 fraction bits,
    normal exponents down to -6, subnormal quantum 2^-9, largest value 448."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    e = np.floor(np.log2(np.where(ax > 0, ax, 1.0)))
    q = 2.0 ** (np.maximum(e, -6.0) - 3.0)
    return np.sign(x) * np.minimum(np.round(ax / q) * q, 448.0)


def _pow2_to_448(amax):
    """The power of two 2^e with the largest e such that amax * 2^e <= 448."""
    amax = np.asarray(amax, dtype=np.float64)
    mant, q = np.frexp(np.where(amax > 0, amax, 1.0))
    e = np.where(mant <= 0.875, 9 - q, 8 - q)
    e = np.clip(np.where(amax > 0, e, 0), -126, 126)
    return 2.0 ** e


def test_pow2_scale_definition():
    """The scale puts the largest magnitude in (224, 448]."""
    amax = np.array([1.0, 0.875, 0.876, 448.0, 449.0, 3e-5, 7.0])
    s = _pow2_to_448(amax)
    assert np.all(amax * s <= 448.0) and np.all(amax * s > 224.0)


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (300, 200, 256), (1000, 77, 100), (5, 3, 16), (700, 900, 192)])
def test_trailing_update_fp8_vs_reference(m, n, k):
    """C - A B with each row of A and each column of B scaled by a power of two
    into the e4m3 range, rounded to e4m3, multiplied in FP32 and unscaled:
    products of two e4m3 values are exact in FP32 and the scales are exact, so
    the only difference from the exact sum of the same products is the FP32
    accumulation."""
    import torch

    import paper_1611_06365_gb300 as lu
    A = li.uniform(m, k, seed=11 + m)
    B = li.uniform(k, n, seed=12 + n)
    C = li.uniform(m, n, seed=13 + k)
    A[0, :] *= 1e-3                                   # rows and columns of different magnitudes
    B[:, 0] *= 37.0
    dA = li.to_device_colmajor(A, dev(), torch.float32)
    dB = li.to_device_colmajor(B, dev(), torch.float32)
    dC = li.to_device_colmajor(C, dev(), torch.float32)
    lu.lu_trailing_update(lu.LU_UPDATE_FP8, dA, dB, dC, m, n, k)
    torch.cuda.synchronize()
    got = li.from_device_colmajor(dC, m)
    A32 = A.astype(np.float32).astype(np.float64)
    B32 = B.astype(np.float32).astype(np.float64)
    C32 = C.astype(np.float32).astype(np.float64)
    sa = _pow2_to_448(np.max(np.abs(A32), axis=1))
    sb = _pow2_to_448(np.max(np.abs(B32), axis=0))
    qa = _e4m3(A32 * sa[:, None])
    qb = _e4m3(B32 * sb[None, :])
    prod = (qa @ qb) / sa[:, None] / sb[None, :]
    mag = (np.abs(qa) @ np.abs(qb)) / sa[:, None] / sb[None, :]
    ref = C32 - prod
    bound = k * 2.0 ** -23 * mag + 2.0 ** -23 * np.abs(ref) + 1e-30
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)
    # e4m3 keeps 4 significant bits: the product is within 2^-3 of the FP32 one, relative to |A||B|
    assert np.max(np.abs(prod - A32 @ B32) / (np.abs(A32) @ np.abs(B32) + 1e-30)) <= 2.0 ** -3


def test_trailing_update_native_fp32():
    import torch

    import paper_1611_06365_gb300 as lu
    m, n, k = 257, 129, 48
    A, B, C = li.uniform(m, k, seed=4), li.uniform(k, n, seed=5), li.uniform(m, n, seed=6)
    dA, dB, dC = (li.to_device_colmajor(X, dev(), torch.float32) for X in (A, B, C))
    lu.lu_trailing_update(lu.LU_UPDATE_NATIVE, dA, dB, dC, m, n, k)
    torch.cuda.synchronize()
    ref = C.astype(np.float32).astype(float) - A.astype(np.float32).astype(float) @ B.astype(np.float32).astype(float)
    assert np.max(np.abs(li.from_device_colmajor(dC, m) - ref)) <= k * 2.0 ** -22 * 2


def _mixed(A, B, **kw):
    import torch

    import paper_1611_06365_gb300 as lu
    n, nrhs = B.shape
    dA = li.to_device_colmajor(A, dev())
    dB = li.to_device_colmajor(B, dev())
    dX = torch.zeros_like(dB)
    rep = lu.lu_solve_mixed(dA, dB, dX, n, **kw)
    torch.cuda.synchronize()
    return li.from_device_colmajor(dX, n), rep


@pytest.mark.parametrize("nrhs", [1, 8])
def test_mixed_uniform_reaches_1e14(oracle_mod, nrhs):
    n = 1500
    A = li.uniform(n, n, seed=li.BASE_SEED + 2000)
    B = li.uniform(n, nrhs, seed=li.BASE_SEED + 2001)
    X, rep = _mixed(A, B, fallback_ratio=-1.0)
    eta = oracle_mod.backward_error(A, X, B)
    assert eta <= 1e-14 and rep.backward_error <= 1e-14
    assert rep.fell_back == 0
    Xo = oracle_mod.getrs(*oracle_mod.getrf(A, nthreads=oracle_mod.default_threads())[:2], B)
    assert np.max(np.abs(X - Xo)) / np.max(np.abs(Xo)) <= 1e-9


@pytest.mark.parametrize("kappa,rung_max", [(1e2, 0), (1e5, 1), (1e8, 2)])
def test_mixed_kappa_ladder(oracle_mod, kappa, rung_max):
    n = 600
    A = li.kappa_matrix(n, kappa, seed=li.BASE_SEED + 2100, k=n)
    xt = li.uniform(n, 1, seed=9)
    xt[:, 0] = 1.0
    B = A @ xt
    X, rep = _mixed(A, B, fallback_ratio=-1.0)
    eta = oracle_mod.backward_error(A, X, B)
    assert eta <= 1e-14, (rep.as_dict(), eta)
    assert rep.rung <= rung_max
    # forward error within kappa * eta (with a safety factor)
    fwd = np.max(np.abs(X - xt)) / np.max(np.abs(xt))
    assert fwd <= 100 * kappa * max(eta, 1e-16)
    # the report's estimate (size of the last correction): the error left is below it,
    # up to the attainable accuracy kappa * eps of an FP64 residual
    est = rep.forward_error_est
    assert np.isfinite(est) and est > 0.0
    assert fwd <= 10 * max(est, kappa * np.finfo(float).eps), (fwd, est)


@pytest.mark.parametrize("kind,rung_max", [("dominant", 0), ("kappa10", 1), ("kappa1e3", 2)])
def test_mixed_fp8_update(oracle_mod, kind, rung_max):
    """With the FP8 update (4 significant bits per operand) the FP32 factors
    are a weak preconditioner: classic refinement converges on a diagonally
    dominant matrix, GMRES-IR on a kappa = 10 matrix, and a kappa = 1e3 matrix
    may need the FP64 factorization.  Every rung ends at eta <= 1e-14."""
    import paper_1611_06365_gb300 as lu
    n = 600
    if kind == "dominant":
        A = li.diag_dominant(n, seed=li.BASE_SEED + 2140)
    else:
        A = li.kappa_matrix(n, 10.0 if kind == "kappa10" else 1e3, seed=li.BASE_SEED + 2150, k=n)
    B = A @ np.ones((n, 1))
    X, rep = _mixed(A, B, update=lu.LU_UPDATE_FP8, fallback_ratio=-1.0)
    eta = oracle_mod.backward_error(A, X, B)
    assert eta <= 1e-14 and rep.rung <= rung_max, (rep.as_dict(), eta)


def test_mixed_refactors_in_fp32_when_the_tensor_core_factors_stall(oracle_mod):
    """Plain BF16 factors (8 significant bits) of a kappa = 1e5 matrix stall
    classic refinement; the ladder refactors once with the FP32 update and
    converges on rung 0 without GMRES-IR or the FP64 factorization."""
    import paper_1611_06365_gb300 as lu
    n = 1200
    A = li.kappa_matrix(n, 1e5, seed=li.BASE_SEED + 2300, k=n)
    B = A @ np.ones((n, 1))
    X, rep = _mixed(A, B, update=lu.LU_UPDATE_BF16, fallback_ratio=-1.0)
    assert oracle_mod.backward_error(A, X, B) <= 1e-14
    assert rep.f32_refactor == 1 and rep.rung == 0 and rep.fell_back == 0, rep.as_dict()
    X2, rep2 = _mixed(A, B, update=lu.LU_UPDATE_BF16, f32_refactor=-1, fallback_ratio=-1.0)   # without it: a later rung
    assert oracle_mod.backward_error(A, X2, B) <= 1e-14
    assert rep2.f32_refactor == 0 and rep2.rung >= 1


def test_mixed_kappa_1e12_falls_back(oracle_mod):
    n = 400
    A = li.kappa_matrix(n, 1e12, seed=li.BASE_SEED + 2200, k=n)
    B = A @ np.ones((n, 1))
    X, rep = _mixed(A, B)
    assert oracle_mod.backward_error(A, X, B) <= 1e-14
    assert rep.rung in (1, 2)


def test_mixed_forced_fallback_path(oracle_mod):
    n = 300
    A = li.uniform(n, n, seed=5)
    B = li.uniform(n, 2, seed=6)
    X, rep = _mixed(A, B, max_iter=1, allow_gmres=0, tol=1e-300)
    assert rep.fell_back == 1 and rep.rung == 2
    assert oracle_mod.backward_error(A, X, B) <= 1e-15


def test_mixed_condition_estimate_and_hopeless_matrices(oracle_mod):
    """The report's condition estimate grows with kappa (a lower estimate, from one
    random right-hand side); with the cost model on, a matrix far too ill-conditioned
    for FP32 factors skips the FP32 refactorization and GMRES-IR once classic
    refinement stalls, and the FP64 fallback reaches the target."""
    n = 400
    ests = []
    for kappa in (1e2, 1e6):
        A = li.kappa_matrix(n, kappa, seed=li.BASE_SEED + 2500, k=n)
        _, rep = _mixed(A, A @ np.ones((n, 1)), fallback_ratio=-1.0)
        ests.append(rep.cond_est)
    assert 1.0 <= ests[0] < ests[1] and ests[1] > 100 * ests[0], ests
    A = li.kappa_matrix(n, 1e12, seed=li.BASE_SEED + 2200, k=n)
    B = A @ np.ones((n, 1))
    X, rep = _mixed(A, B, fallback_ratio=1e9)   # a generous budget: only the condition rule can stop
    assert rep.cond_est * np.finfo(np.float32).eps > 16
    assert rep.rung == 2 and rep.cost_stop == 1 and rep.f32_refactor == 0 and rep.gmres_iters == 0, rep.as_dict()
    assert oracle_mod.backward_error(A, X, B) <= 1e-14


def test_mixed_cost_model_takes_the_fallback_when_refinement_would_cost_more(oracle_mod):
    """With the FP64 fallback predicted to cost next to nothing, the ladder stops
    refining as soon as it has a contraction rate to predict from, skips the
    FP32 refactorization and GMRES-IR, and the fallback reaches the target."""
    import paper_1611_06365_gb300 as lu
    n = 1200
    A = li.kappa_matrix(n, 1e5, seed=li.BASE_SEED + 2300, k=n)
    B = A @ np.ones((n, 1))
    X, rep = _mixed(A, B, update=lu.LU_UPDATE_BF16, fallback_ratio=1e-6)
    assert rep.cost_stop == 1 and rep.rung == 2 and rep.fell_back == 1, rep.as_dict()
    assert rep.f32_refactor == 0 and rep.gmres_iters == 0 and rep.t_fallback_ms > 0.0
    assert oracle_mod.backward_error(A, X, B) <= 1e-14


@pytest.mark.parametrize("nrhs", [1, 3])
def test_mixed_cost_model_generous_budget_changes_nothing(nrhs):
    """A fallback predicted to cost far more than any refinement leaves the ladder
    as it is without the cost model: the same rungs and the same bits."""
    import paper_1611_06365_gb300 as lu
    n = 1200
    A = li.kappa_matrix(n, 1e5, seed=li.BASE_SEED + 2300, k=n)
    B = A @ li.uniform(n, nrhs, seed=77)
    X1, r1 = _mixed(A, B, update=lu.LU_UPDATE_BF16, fallback_ratio=-1.0)
    X2, r2 = _mixed(A, B, update=lu.LU_UPDATE_BF16, fallback_ratio=1e12)
    assert r2.cost_stop == 0
    assert (r1.rung, r1.iterations, r1.gmres_iters, r1.f32_refactor) == (r2.rung, r2.iterations, r2.gmres_iters,
                                                                          r2.f32_refactor)
    assert np.array_equal(X1, X2)


def test_mixed_gmres_columns_together_match_alone(oracle_mod):
    """GMRES-IR iterates the right-hand side columns side by side, each with its
    own basis and stopping decisions: every column of a 5-column solve reaches
    the target, as when solved alone."""
    import paper_1611_06365_gb300 as lu
    n = 700
    A = li.kappa_matrix(n, 1e3, seed=li.BASE_SEED + 2400, k=n)   # kappa * 2^-8 ~ 4: classic refinement stalls
    B = A @ li.uniform(n, 5, seed=78)
    X, rep = _mixed(A, B, update=lu.LU_UPDATE_BF16, f32_refactor=-1, allow_fallback=0, fallback_ratio=-1.0)
    assert rep.rung == 1 and rep.gmres_iters > 0, rep.as_dict()
    for q in range(5):
        assert oracle_mod.backward_error(A, X[:, q:q + 1], B[:, q:q + 1]) <= 1e-14, q
        Xq, rq = _mixed(A, B[:, q:q + 1], update=lu.LU_UPDATE_BF16, f32_refactor=-1, allow_fallback=0,
                        fallback_ratio=-1.0)
        assert rq.rung == 1 and oracle_mod.backward_error(A, Xq, B[:, q:q + 1]) <= 1e-14
