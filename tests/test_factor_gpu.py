"""Parity of the CUDA factorization (lu_factor) with the CPU oracle.

Bar (FP64 path): the pivot vector equals the oracle's bit for bit,
||PA - LU||_F / ||A||_F <= 10 n eps64, and every entry of the packed factors
is within 10 n eps64 max|LU| of the oracle's (the two differ only in rounding:
FMA and blocked summation order on the GPU, two roundings per update in the
oracle).  Exact families (dyadic P^T L U, Wilkinson) must match bit for bit
on every path.
"""
import numpy as np
import pytest

import lu_inputs as li
from tests._parity import oracle_parity
from tests.gpu_util import EPS32, EPS64, expected_ipiv, factor_gpu

pytestmark = pytest.mark.gpu


def _parity_f64(oracle_mod, A, **opts):
    n = A.shape[0]
    LU, ipiv, info, _, _ = factor_gpu(A, "f64", **opts)
    infoo = oracle_mod.getrf(A)[2]
    assert info == infoo
    # whole pivot vector, near-tie rule (tests/_parity.py)
    LUo, _ = oracle_parity(oracle_mod, A, ipiv)
    r, a = oracle_mod.lu_residual_fro(A, LU, ipiv)
    assert r / a <= 10 * n * EPS64
    assert np.max(np.abs(LU - LUo)) <= 10 * n * EPS64 * max(1.0, np.max(np.abs(LUo)))
    return LU, ipiv


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 65, 100, 257, 512, 700])
def test_f64_uniform_matches_oracle(oracle_mod, n):
    A = li.uniform(n, n, seed=li.BASE_SEED + n)
    _parity_f64(oracle_mod, A)


def test_f64_c1_workload_n512(oracle_mod):
    """n = 512, lda = 512, entries uniform [-1, 1), seed of the small workload."""
    A = li.uniform(512, 512, seed=li.BASE_SEED + 1000)
    _parity_f64(oracle_mod, A)


@pytest.mark.parametrize("nb,nb_inner", [(16, 16), (32, 8), (48, 16), (64, 32)])
def test_f64_block_sizes_ragged(oracle_mod, nb, nb_inner):
    A = li.uniform(333, 333, seed=7)
    _parity_f64(oracle_mod, A, nb=nb, nb_inner=nb_inner)


def test_f64_lda_padding(oracle_mod):
    A = li.uniform(150, 150, seed=8)
    LU, ipiv, info, dA, _ = factor_gpu(A, "f64", ld=173)
    pivo = oracle_mod.getrf(A)[1]
    assert np.array_equal(ipiv, pivo)
    assert float(dA[:, 150:].abs().sum()) == 0.0      # padding untouched


def test_schedule_invariance_bits():
    """Look-ahead on/off and panel cluster sizes change the schedule, not the arithmetic."""
    A = li.uniform(600, 600, seed=9)
    ref, piv_ref, _, _, _ = factor_gpu(A, "f64", nb=32, lookahead=-1, panel_ctas=16)
    for la, ctas, tile in ((1, 16, 0), (1, 4, 0), (-1, 2, 0), (1, 1, 0), (1, 8, 1), (1, 8, 2), (2, 8, 2)):
        LU, ipiv, _, _, _ = factor_gpu(A, "f64", nb=32, lookahead=la, panel_ctas=ctas, tile=tile)
        assert np.array_equal(ipiv, piv_ref)
        assert np.array_equal(LU, ref), (la, ctas, tile)


@pytest.mark.parametrize("dtype,update", [("f64", 0), ("f32", 0), ("f32", 1), ("f32", 2), ("f32", 3)])
@pytest.mark.parametrize("n", [40, 300, 1030])
def test_dyadic_exact_all_paths(n, dtype, update):
    """L entries k/8 and U integers in [-8, 8] are exact in FP64, FP32, BF16
    and e4m3, so every path, the FP8 update included, recovers P, L, U exactly
    (for FP8 this also shows that the tensor cores accumulate these products
    exactly in FP32)."""
    A, perm, L, U = li.dyadic_plu(n, seed=500 + n)
    LU, ipiv, info, _, _ = factor_gpu(A, dtype, update=update)
    assert info == 0
    assert np.array_equal(ipiv, expected_ipiv(perm))
    L2 = np.tril(LU, -1) + np.eye(n)
    U2 = np.triu(LU)
    assert np.array_equal(L2, L) and np.array_equal(U2, U)


@pytest.mark.parametrize("dtype,n", [("f64", 64), ("f64", 500), ("f32", 100)])
def test_wilkinson_growth(dtype, n):
    LU, ipiv, info, _, _ = factor_gpu(li.wilkinson(n), dtype)
    assert np.array_equal(ipiv, np.arange(1, n + 1))          # all ties -> first index
    assert np.array_equal(LU[:, n - 1], 2.0 ** np.arange(n))   # growth 2^(n-1)


def test_singular_info_and_completion(oracle_mod):
    n = 90
    A = li.uniform(n, n, seed=12)
    A[:, 37] = 0.0                       # column 37 is zero: first zero pivot at step 37 at the latest
    LU, ipiv, info, _, _ = factor_gpu(A, "f64")
    LUo, pivo, infoo = oracle_mod.getrf(A)
    assert infoo > 0 and info == infoo
    assert np.array_equal(ipiv, pivo)
    B = np.zeros((n, n))                 # all-zero matrix: info = 1, no interchanges
    LU, ipiv, info, _, _ = factor_gpu(B, "f64")
    assert info == 1 and np.array_equal(ipiv, np.arange(1, n + 1)) and not LU.any()


def test_diag_dominant_no_interchange():
    A = li.diag_dominant(400, seed=3)
    _, ipiv, _, _, _ = factor_gpu(A, "f64")
    assert np.array_equal(ipiv, np.arange(1, 401))


def test_f32_native_backward_error(oracle_mod):
    n = 800
    A = li.uniform(n, n, seed=14)
    LU, ipiv, info, _, _ = factor_gpu(A, "f32")
    r, a = oracle_mod.lu_residual_fro(A.astype(np.float32).astype(np.float64), LU, ipiv)
    assert r / a <= 10 * n * EPS32
    assert np.max(np.abs(np.tril(LU, -1))) <= 1.0     # valid partial pivoting


def test_f32_bf16_update_backward_error(oracle_mod):
    """BF16 operands in the trailing update: P A = L U + E with the standard
    componentwise bound |E| <= c u |L||U|, u = 2^-8 for the two BF16 roundings
    of each product (the FP32 parts contribute far less).  The pivots must form
    a valid partial-pivoting sequence for the computed Schur complements
    (|l_ij| <= 1)."""
    n = 1100
    A = li.uniform(n, n, seed=15)
    LU, ipiv, info, _, _ = factor_gpu(A, "f32", update=1)
    A32 = A.astype(np.float32).astype(np.float64)
    r, a = oracle_mod.lu_residual_fro(A32, LU, ipiv)
    L, U = oracle_mod.unpack(LU)
    growth = np.linalg.norm(np.abs(L) @ np.abs(U)) / a
    assert r / a <= 2.0 ** -8 * growth
    assert r / a >= 2.0 ** -24          # the BF16 rounding really is there
    assert np.max(np.abs(np.tril(LU, -1))) <= 1.0


def test_f32_bf16x3_update_backward_error(oracle_mod):
    """Split BF16 (three products): the update keeps about 16 bits, so the
    bound of the BF16 case tightens to u = 2^-16; still a valid pivoting."""
    n = 1100
    A = li.uniform(n, n, seed=15)
    LU, ipiv, info, _, _ = factor_gpu(A, "f32", update=2)
    A32 = A.astype(np.float32).astype(np.float64)
    r, a = oracle_mod.lu_residual_fro(A32, LU, ipiv)
    L, U = oracle_mod.unpack(LU)
    growth = np.linalg.norm(np.abs(L) @ np.abs(U)) / a
    assert r / a <= 2.0 ** -16 * growth
    assert np.max(np.abs(np.tril(LU, -1))) <= 1.0


@pytest.mark.parametrize("update", [1, 2, 3])
def test_f32_tc_update_large_lookahead_invariance(update):
    """The tensor-core path under look-ahead on and off gives identical bits."""
    A = li.uniform(2304, 2304, seed=16)
    ref, pref, _, _, _ = factor_gpu(A, "f32", update=update, lookahead=-1)
    for depth, share in ((1, 0), (2, 0), (4, 0), (1, -1), (2, -1)):
        got, pgot, _, _, _ = factor_gpu(A, "f32", update=update, lookahead=depth, sm_share=share)
        assert np.array_equal(pref, pgot) and np.array_equal(ref, got), (depth, share)


@pytest.mark.parametrize("depth", [2, 3, 4])
def test_deeper_lookahead_same_bits_and_oracle_pivots(oracle_mod, depth):
    """Look-ahead of depth d (the panel branch keeps d strips current) reorders
    the schedule only: the factors are bit-identical to depth 1 and to no
    look-ahead, and the pivots equal the oracle's; ragged last strips included."""
    A = li.uniform(1000, 1000, seed=23)
    ref, piv_ref, _, _, _ = factor_gpu(A, "f64", nb=32, lookahead=-1)
    got, piv, info, _, _ = factor_gpu(A, "f64", nb=32, lookahead=depth)
    assert info == 0 and np.array_equal(piv, piv_ref) and np.array_equal(got, ref)
    oracle_parity(oracle_mod, A, piv)
    B = li.uniform(777, 777, seed=24)
    ref, piv_ref, _, _, _ = factor_gpu(B, "f64", nb=48, lookahead=1)
    got, piv, _, _, _ = factor_gpu(B, "f64", nb=48, lookahead=depth)
    assert np.array_equal(piv, piv_ref) and np.array_equal(got, ref)


def test_empty_matrix():
    import torch

    import paper_1611_06365_gb300 as lu
    dA = torch.zeros((1, 1), dtype=torch.float64, device="cuda:0")
    ipiv = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    info = torch.full((1,), 5, dtype=torch.int32, device="cuda:0")
    lu.lu_factor(dA, ipiv, info, 0)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
