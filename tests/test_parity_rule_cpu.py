"""The near-tie rule of the pivot parity checks, exercised on the CPU.

The "other implementation" here is the oracle itself with a choice planted
on the oracle side (a forced pivot), so the rule's three outcomes are seen
without a GPU: exact agreement, an accepted tie followed by a forced re-run
that agrees, and a rejected mismatch at a clear gap.
"""
import numpy as np
import pytest

import lu_inputs as li
from tests._parity import golden_agreement, oracle_parity, tie_bound


def _tied_matrix(n=40, seed=3):
    """Uniform matrix whose first column has an exact magnitude tie between its
    two largest entries (rows 5 and 11, opposite signs): the search takes row 5."""
    A = li.uniform(n, n, seed)
    A[:, 0] *= 0.5
    A[5, 0], A[11, 0] = 0.75, -0.75
    return A


def test_identical_pivots_need_no_rerun(oracle_mod):
    A = li.uniform(64, 64, 1)
    _, piv, _ = oracle_mod.getrf(A)
    LUo, reruns = oracle_parity(oracle_mod, A, piv)
    assert reruns == []


def test_tie_is_rerun_with_the_other_choice(oracle_mod):
    A = _tied_matrix()
    _, piv, _, gaps = oracle_mod.getrf(A, want_gaps=True)
    assert piv[0] == 6 and gaps[0] == 0.0
    forced = np.zeros(A.shape[0], dtype=np.int32)
    forced[0] = 12                                   # the equally large row 11 (1-based 12)
    LU_other, piv_other, _ = oracle_mod.getrf(A, forced=forced)
    LUo, reruns = oracle_parity(oracle_mod, A, piv_other)
    assert reruns == [(0, 0.0)]
    assert np.array_equal(LUo, LU_other)


def test_clear_mismatch_fails(oracle_mod):
    A = li.uniform(48, 48, 2)
    _, piv, _, gaps = oracle_mod.getrf(A, want_gaps=True)
    assert gaps[0] > tie_bound(48)
    forced = np.zeros(48, dtype=np.int32)
    forced[0] = piv[0] % 48 + 1                      # any other row
    _, piv_wrong, _ = oracle_mod.getrf(A, forced=forced)
    with pytest.raises(AssertionError, match="pivot mismatch at step 0"):
        oracle_parity(oracle_mod, A, piv_wrong)


def test_golden_agreement_summary():
    g = np.arange(1, 11, dtype=np.int32)
    assert golden_agreement(g, g, {}, 10)["pivot_agreement"] == 1.0
    h = g.copy()
    h[4] = 9
    out = golden_agreement(h, g, {4: 1e-15}, 10)
    assert out["first_mismatch_step"] == 4 and out["tie_ambiguous"] and out["pivot_agreement"] == 0.9
    out = golden_agreement(h, g, {}, 10)
    assert out["first_mismatch_gap"] is None and not out["tie_ambiguous"]
