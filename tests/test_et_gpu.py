"""Early termination of the panel factorization (section 4.2, Figure LU_LA_ET).

With lu_opts.early_term = 1 the panel of step k+1 stops at the end of the
inner panel during which the remainder update of step k finished, and step
k+1 has the width the panel reached.  The blocking changes, the elimination
does not: the pivots follow the oracle's (near-tie rule), exact families stay
exact on every update path, and the reported panel widths tile the matrix.
early_term = 2 stops every panel at its first inner boundary: a fixed
schedule through the same code, so its widths are known in advance.
"""
import numpy as np
import pytest

import lu_inputs as li
from tests._parity import oracle_parity
from tests.gpu_util import EPS64, expected_ipiv, factor_gpu

pytestmark = pytest.mark.gpu


def _widths():
    import paper_1611_06365_gb300 as lu
    return lu.lu_last_panel_widths()


def _check_f64(oracle_mod, A, LU, ipiv, info):
    n = A.shape[0]
    assert info == 0
    LUo, _ = oracle_parity(oracle_mod, A, ipiv)
    r, a = oracle_mod.lu_residual_fro(A, LU, ipiv)
    assert r / a <= 10 * n * EPS64
    assert np.max(np.abs(LU - LUo)) <= 10 * n * EPS64 * max(1.0, float(np.max(np.abs(LUo))))


def test_forced_stops_give_known_widths_and_oracle_pivots(oracle_mod):
    """Panel 0 runs whole (no update runs beside it); every later panel stops
    after its first inner panel of 16 columns; the last one (a single inner
    panel) runs whole: 700 = 64 + 39 * 16 + 12."""
    n = 700
    A = li.uniform(n, n, seed=li.BASE_SEED + 41)
    LU, ipiv, info, _, _ = factor_gpu(A, "f64", nb=64, nb_inner=16, early_term=2)
    assert _widths() == [64] + [16] * 39 + [12]
    _check_f64(oracle_mod, A, LU, ipiv, info)


def test_without_early_termination_widths_are_nominal():
    A = li.uniform(300, 300, seed=42)
    factor_gpu(A, "f64", nb=64, nb_inner=16)
    assert _widths() == [64, 64, 64, 64, 44]


@pytest.mark.parametrize("n", [1000, 2049])
def test_adaptive_stops_keep_oracle_pivots(oracle_mod, n):
    """Where the panels stop depends on timing; whatever it was, the widths tile
    the matrix in whole inner panels and the pivots are the oracle's."""
    A = li.uniform(n, n, seed=li.BASE_SEED + 43 + n)
    LU, ipiv, info, _, _ = factor_gpu(A, "f64", nb=64, nb_inner=16, early_term=1)
    w = _widths()
    assert sum(w) == n and w[0] == 64
    assert all(x % 16 == 0 or i == len(w) - 1 for i, x in enumerate(w))
    _check_f64(oracle_mod, A, LU, ipiv, info)


def test_adaptive_emulated_update_keeps_oracle_pivots(oracle_mod):
    import paper_1611_06365_gb300 as lu
    n = 1100
    A = li.uniform(n, n, seed=li.BASE_SEED + 44)
    LU, ipiv, info, _, _ = factor_gpu(A, "f64", nb=64, nb_inner=16, early_term=1, update=lu.LU_UPDATE_F64EMU)
    assert sum(_widths()) == n
    _check_f64(oracle_mod, A, LU, ipiv, info)


@pytest.mark.parametrize("dtype,update", [("f64", 0), ("f64", 4), ("f32", 0), ("f32", 1), ("f32", 2), ("f32", 3)])
@pytest.mark.parametrize("et", [1, 2])
def test_early_termination_exact_on_dyadic(dtype, update, et):
    """Dyadic P^T L U is recovered exactly whatever the blocking, so any step
    applied to the wrong columns, rows or width breaks the equality; the
    staged operands of the tensor-core updates (K padded past the factored
    width) included."""
    n = 530
    A, perm, L, U = li.dyadic_plu(n, seed=570 + update)
    LU, ipiv, info, _, _ = factor_gpu(A, dtype, nb=64, nb_inner=16, early_term=et, update=update)
    assert info == 0
    assert sum(_widths()) == n
    assert np.array_equal(ipiv, expected_ipiv(perm))
    assert np.array_equal(np.tril(LU, -1) + np.eye(n), L) and np.array_equal(np.triu(LU), U)


def test_forced_split_bf16_matches_its_own_accuracy(oracle_mod):
    """The FP32 factorization with the split-BF16 update and forced stops keeps
    the update's accuracy (backward error of the FP32-rounded input)."""
    n = 1100
    A = li.uniform(n, n, seed=45)
    LU, ipiv, info, _, _ = factor_gpu(A, "f32", nb=64, nb_inner=16, early_term=2, update=2)
    assert info == 0
    A32 = A.astype(np.float32).astype(np.float64)
    r, a = oracle_mod.lu_residual_fro(A32, LU, ipiv)
    L, U = oracle_mod.unpack(LU)
    growth = np.linalg.norm(np.abs(L) @ np.abs(U)) / a
    assert r / a <= 2.0 ** -16 * growth
    assert np.max(np.abs(np.tril(LU, -1))) <= 1.0
