"""The emulated FP64 trailing update (LU_UPDATE_F64EMU): FP64 operands split
into seven BF16 digit slices below power-of-two row / column scales, 28 slice
products on the tensor cores, one FP64 rounding per element.

Checked against a reference in extended precision (numpy longdouble: the
products of two doubles and their sums carry at least 64 significand bits),
element by element: the emulated error must stay within a few FP64 roundings
of each result plus 2^-50 of the row and column scales' product, and below
the error of the plain DFMA update on the same data.  The factorization with
this update is compared with the oracle like the plain FP64 path (whole pivot
vector, near-tie rule) and must recover the exact dyadic family exactly.
"""
import numpy as np
import pytest

import lu_inputs as li
from tests._parity import oracle_parity
from tests.gpu_util import EPS64, dev, expected_ipiv, factor_gpu

pytestmark = pytest.mark.gpu


def _update(update, A, B, C):
    import torch

    import paper_1611_06365_gb300 as lu
    m, k = A.shape
    n = B.shape[1]
    dA = li.to_device_colmajor(A, dev())
    dB = li.to_device_colmajor(B, dev())
    dC = li.to_device_colmajor(C, dev())
    lu.lu_trailing_update_f64(update, dA, dB, dC, m, n, k)
    torch.cuda.synchronize()
    return li.from_device_colmajor(dC, m)


def _reference(A, B, C):
    Al, Bl, Cl = (x.astype(np.longdouble) for x in (A, B, C))
    return Cl - Al @ Bl


@pytest.mark.parametrize("m,n,k", [(300, 200, 64), (129, 33, 17), (1000, 257, 32), (64, 1, 1), (517, 700, 64)])
def test_f64emu_update_accuracy(m, n, k):
    import paper_1611_06365_gb300 as lu
    rng = np.random.default_rng(m * 7 + n + k)
    A = li.uniform(m, k, seed=m + k)
    B = li.uniform(k, n, seed=n + 3 * k) * 10.0 ** rng.integers(-3, 4, size=(1, n))   # columns of mixed scale
    C = li.uniform(m, n, seed=m + n)
    ref = _reference(A, B, C)
    emu = _update(lu.LU_UPDATE_F64EMU, A, B, C)
    nat = _update(lu.LU_UPDATE_NATIVE, A, B, C)
    err_emu = np.abs(emu.astype(np.longdouble) - ref).astype(np.float64)
    err_nat = np.abs(nat.astype(np.longdouble) - ref).astype(np.float64)
    # the row and column scales 2^e_i 2^e_j are below 4 max|A(i,:)| max|B(:,j)|; the
    # dropped digit pairs and the rounding of the shared sixth accumulator stay below
    # 2^-48.5 of them in the worst case (a K-term DFMA chain: K^2 2^-53)
    scale = np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :]
    bound = 2 * EPS64 * np.abs(ref.astype(np.float64)) + 2.0 ** -46 * scale
    assert np.all(err_emu <= bound), float(np.max(err_emu / bound))
    assert np.max(err_emu) <= max(np.max(err_nat), 4 * EPS64 * float(np.max(np.abs(ref.astype(np.float64)))))


def test_f64emu_update_extreme_column_scales():
    """Columns of B near the top of the FP64 range (scale 2^970: the column scale is
    applied by an FP64 multiply) and in the subnormal range (the same), beside
    ordinary and tiny normal columns (applied by adding to the exponent): every
    element within the accuracy bound of the extended-precision reference."""
    import paper_1611_06365_gb300 as lu
    m, n, k = 300, 6, 64
    A = li.uniform(m, k, seed=11)
    B = li.uniform(k, n, seed=12)
    B[:, 0] *= 2.0 ** 970
    B[:, 1] *= 2.0 ** -1040          # subnormal entries
    B[:, 2] *= 2.0 ** -1000
    B[:, 3] *= 2.0 ** 900
    C = li.uniform(m, n, seed=13)
    C[:, 0] *= 2.0 ** 970
    C[:, 3] *= 2.0 ** 900
    ref = _reference(A, B, C)
    emu = _update(lu.LU_UPDATE_F64EMU, A, B, C)
    err = np.abs(emu.astype(np.longdouble) - ref)
    scale = (np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :]).astype(np.longdouble)
    bound = 2 * EPS64 * np.abs(ref) + np.longdouble(2.0 ** -46) * scale + np.longdouble(2.0 ** -1074)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert np.all(np.isfinite(emu))


def test_f64emu_update_exact_on_dyadic_operands():
    """Operands with few significant bits (multiples of 1/8 below 8) give exact products:
    the result equals the exactly rounded one bit for bit."""
    import paper_1611_06365_gb300 as lu
    m, n, k = 256, 96, 64
    h = li.splitmix64(77, np.arange(m * k + k * n, dtype=np.uint64))
    A = ((h[:m * k] % np.uint64(127)).astype(np.float64) - 63.0).reshape(m, k) / 8.0
    B = ((h[m * k:] % np.uint64(127)).astype(np.float64) - 63.0).reshape(k, n) / 8.0
    C = li.uniform(m, n, seed=5)
    ref = (C.astype(np.longdouble) - A.astype(np.longdouble) @ B.astype(np.longdouble)).astype(np.float64)
    assert np.array_equal(_update(lu.LU_UPDATE_F64EMU, A, B, C), ref)


def test_f64emu_dyadic_factorization_exact():
    import paper_1611_06365_gb300 as lu
    for n in (40, 300, 1030):
        A, perm, L, U = li.dyadic_plu(n, seed=500 + n)
        LU, ipiv, info, _, _ = factor_gpu(A, "f64", update=lu.LU_UPDATE_F64EMU)
        assert info == 0
        assert np.array_equal(ipiv, expected_ipiv(perm))
        assert np.array_equal(np.tril(LU, -1) + np.eye(n), L) and np.array_equal(np.triu(LU), U)


@pytest.mark.parametrize("n", [700, 2049])
def test_f64emu_factorization_matches_oracle(oracle_mod, n):
    import paper_1611_06365_gb300 as lu
    A = li.uniform(n, n, seed=li.BASE_SEED + 3 * n)
    LU, ipiv, info, _, _ = factor_gpu(A, "f64", update=lu.LU_UPDATE_F64EMU)
    assert info == 0
    LUo, _ = oracle_parity(oracle_mod, A, ipiv)
    r, a = oracle_mod.lu_residual_fro(A, LU, ipiv)
    assert r / a <= 10 * n * EPS64
    assert np.max(np.abs(LU - LUo)) <= 10 * n * EPS64 * max(1.0, float(np.max(np.abs(LUo))))


def test_f64emu_schedule_invariance_bits():
    """Look-ahead on/off and panel teams change the schedule, not the arithmetic."""
    import paper_1611_06365_gb300 as lu
    A = li.uniform(600, 600, seed=19)
    ref, piv_ref, _, _, _ = factor_gpu(A, "f64", update=lu.LU_UPDATE_F64EMU, nb=64, lookahead=-1)
    for la, ctas, share, tile in ((1, 8, 0, 0), (1, 2, 0, 0), (-1, 4, 0, 0), (2, 8, 0, 0), (3, 4, 0, 0), (1, 8, -1, 0),
                                  (2, 16, -1, 0), (1, 8, 0, 1), (1, 8, 0, 2), (2, 4, -1, 2)):
        LU, ipiv, _, _, _ = factor_gpu(A, "f64", update=lu.LU_UPDATE_F64EMU, nb=64, lookahead=la, panel_ctas=ctas,
                                       sm_share=share, tile=tile)
        assert np.array_equal(ipiv, piv_ref) and np.array_equal(LU, ref), (la, ctas, share, tile)


def test_f64emu_full_size_n8192(oracle_mod):
    """n = 8192 with the default emulated plan: the whole pivot vector against the oracle."""
    import torch

    import paper_1611_06365_gb300 as lu
    n = 8192
    seed = 20161106 + 1000 * 2 + 2
    A = li.uniform_colmajor_torch(n, n, seed, dev(), torch.float64)
    dA = A.clone()
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev())
    info = torch.full((1,), -1, dtype=torch.int32, device=dev())
    lu.lu_factor(dA, ipiv, info, n, update=lu.LU_UPDATE_F64EMU)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    A_f, LU_f = A.cpu().numpy().T, dA.cpu().numpy().T
    LUo, _ = oracle_parity(oracle_mod, np.asfortranarray(A_f), ipiv.cpu().numpy())
    assert np.max(np.abs(LU_f - LUo)) <= 10 * n * EPS64 * max(1.0, float(np.max(np.abs(LUo))))


def test_f64emu_update_nonfinite_propagates():
    """An infinity in a row of A or a NaN in a column of B makes that row or column
    of the result non-finite, as in the DFMA update (the integer sums cannot hold
    them, the infinite scale carries them)."""
    import paper_1611_06365_gb300 as lu
    m, n, k = 200, 70, 40
    A = li.uniform(m, k, seed=3)
    B = li.uniform(k, n, seed=4)
    C = li.uniform(m, n, seed=5)
    A[5, 7] = np.inf
    B[11, 3] = np.nan
    emu = _update(lu.LU_UPDATE_F64EMU, A, B, C)
    nat = _update(lu.LU_UPDATE_NATIVE, A, B, C)
    assert np.array_equal(np.isfinite(emu), np.isfinite(nat))
    assert not np.any(np.isfinite(emu[5, :])) and not np.any(np.isfinite(emu[:, 3]))
    assert np.isfinite(np.delete(np.delete(emu, 5, axis=0), 3, axis=1)).all()
