"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test names what fixes the expected value: a hand-worked example, a
closed form, a textbook property, brute force or exact rational arithmetic.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import lu_inputs as li
from tests._exact import leibniz_det, rational_gepp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    sections, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            toks = line.split()
            if len(toks) == 1 and not toks[0].lstrip("-").replace("/", "").isdigit():
                cur = toks[0]
                sections[cur] = []
            elif cur is None or (toks[0].isalpha() and toks[0] not in sections):
                sections[toks[0]] = toks[1:]
            else:
                sections[cur].append([Fraction(t) for t in toks])
    return sections


def test_3x3_hand_worked(oracle_mod):
    g = _read_golden("lu3x3.txt")
    A = np.array([[float(x) for x in r] for r in g["A"]])
    LU, ipiv, info = oracle_mod.getrf(A)
    assert info == 0
    assert list(ipiv) == [int(x) for x in g["ipiv"][0]]
    L, U = oracle_mod.unpack(LU)
    Lx = np.array([[float(x) for x in r] for r in g["L"]])
    Ux = np.array([[float(x) for x in r] for r in g["U"]])
    # within a few units of roundoff of the exact rationals (each entry is
    # produced by at most three rounded operations on rounded inputs)
    eps = np.finfo(float).eps
    assert np.all(np.abs(L - Lx) <= 4 * eps * np.abs(Lx))
    assert np.all(np.abs(U - Ux) <= 4 * eps * np.abs(Ux))
    assert list(U[0]) == [7.0, 8.0, 10.0] and L[2, 0] == 4.0 / 7.0 and L[1, 0] == 1.0 / 7.0
    det = np.prod(np.diag(U)) * (-1) ** int(np.sum(ipiv != np.arange(1, 4)))
    assert abs(det - float(g["det"][0][0])) < 1e-13


def test_wilkinson_golden_and_closed_form(oracle_mod):
    g = {}
    with open(os.path.join(GOLDEN, "wilkinson_u_lastcol.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                t = line.split()
                g[t[0]] = [int(x) for x in t[1:]]
    n = g["n"][0]
    LU, ipiv, info = oracle_mod.getrf(li.wilkinson(n))
    assert list(ipiv) == g["ipiv"]
    assert list(LU[:, n - 1]) == [float(v) for v in g["u_col_n"]]
    for n in (2, 17, 64, 300):
        LU, ipiv, info = oracle_mod.getrf(li.wilkinson(n))
        assert info == 0
        assert np.array_equal(ipiv, np.arange(1, n + 1))
        assert np.array_equal(LU[:, n - 1], 2.0 ** np.arange(n))   # growth 2^(n-1), exact
        L, U = oracle_mod.unpack(LU)
        assert np.array_equal(np.tril(L, -1), np.tril(-np.ones((n, n)), -1))


def _expected_ipiv(perm):
    """Sequential interchanges that bring row perm[j] of A to position j."""
    n = len(perm)
    cur = list(range(n))          # cur[position] = original row
    where = {r: r for r in range(n)}
    ipiv = []
    for j in range(n):
        p = where[perm[j]]
        ipiv.append(p + 1)
        rj, rp = cur[j], cur[p]
        cur[j], cur[p] = rp, rj
        where[rp], where[rj] = j, p
    return np.array(ipiv)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33, 100, 257])
def test_dyadic_plu_exact(oracle_mod, n):
    A, perm, L, U = li.dyadic_plu(n, seed=1000 + n)
    LU, ipiv, info = oracle_mod.getrf(A, nthreads=3)
    assert info == 0
    assert np.array_equal(ipiv, _expected_ipiv(perm))
    L2, U2 = oracle_mod.unpack(LU)
    assert np.array_equal(L2, L) and np.array_equal(U2, U)


def test_dyadic_solve_exact(oracle_mod):
    n = 120
    A, perm, L, U = li.dyadic_plu(n, seed=77)
    x_true = ((li.splitmix64(5, np.arange(n, dtype=np.uint64)) % np.uint64(9)).astype(np.int64) - 4).astype(float)
    b = A @ x_true                     # integers times multiples of 1/8: exact
    LU, ipiv, info = oracle_mod.getrf(A)
    x = oracle_mod.getrs(LU, ipiv, b)
    assert np.array_equal(x, x_true)


@pytest.mark.parametrize("seed", range(12))
def test_leibniz_determinant(oracle_mod, seed):
    n = 2 + seed % 6                                   # 2..7
    h = li.splitmix64(900 + seed, np.arange(n * n, dtype=np.uint64))
    Ai = ((h % np.uint64(19)).astype(np.int64) - 9).reshape(n, n)
    det = leibniz_det(Ai.tolist())
    LU, ipiv, info = oracle_mod.getrf(Ai.astype(float))
    if det == 0:
        return
    assert info == 0
    nswap = int(np.sum(ipiv != np.arange(1, n + 1)))
    d = np.prod(np.diag(LU)) * (-1) ** nswap
    assert abs(d - float(det)) <= 1e-12 * max(1.0, abs(float(det)))


@pytest.mark.parametrize("seed", range(10))
def test_exact_rational_pivots(oracle_mod, seed):
    n = 3 + seed % 8                                   # 3..10
    h = li.splitmix64(4000 + seed, np.arange(n * n, dtype=np.uint64))
    Ai = ((h % np.uint64(2001)).astype(np.int64) - 1000).reshape(n, n)
    ipiv_x, Lx, Ux = rational_gepp(Ai.tolist())
    LU, ipiv, info = oracle_mod.getrf(Ai.astype(float))
    assert list(ipiv) == ipiv_x
    L, U = oracle_mod.unpack(LU)
    Lf = np.array([[float(v) for v in r] for r in Lx])
    Uf = np.array([[float(v) for v in r] for r in Ux])
    scale = np.max(np.abs(Uf))
    assert np.max(np.abs(L - Lf)) <= 1e-12
    assert np.max(np.abs(U - Uf)) <= 1e-12 * scale


def test_column_dominant_no_interchange(oracle_mod):
    for n in (5, 64, 200):
        LU, ipiv, info = oracle_mod.getrf(li.diag_dominant(n, seed=n))
        assert np.array_equal(ipiv, np.arange(1, n + 1))


def test_zero_pivot_info_and_continue(oracle_mod):
    A = np.array([[0.0, 1.0, 2.0], [0.0, 2.0, 1.0], [0.0, 4.0, 3.0]])
    LU, ipiv, info = oracle_mod.getrf(A)
    assert info == 1                      # first zero pivot, 1-based
    # step 0: all-zero column, first index -> no interchange, nothing scaled;
    # step 1: largest |a_i1| among rows 1..2 is 4 -> ipiv[1] = 3
    assert list(ipiv) == [1, 3, 2] or list(ipiv) == [1, 3, 3]
    assert list(ipiv)[:2] == [1, 3]
    assert np.array_equal(LU[:, 0], [0.0, 0.0, 0.0])
    # rank-2 singular matrix: the second zero pivot does not overwrite info
    B = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [3.0, 6.0, 9.0]])
    LU, ipiv, info = oracle_mod.getrf(B)
    assert info == 2


def test_threads_do_not_change_bits(oracle_mod):
    A = li.uniform(301, seed=9)
    r1 = oracle_mod.getrf(A, nthreads=1)
    for t in (2, 5, 8):
        rt = oracle_mod.getrf(A, nthreads=t)
        assert np.array_equal(r1[0], rt[0]) and np.array_equal(r1[1], rt[1])


def test_random_backward_stable(oracle_mod):
    n = 200
    A = li.uniform(n, seed=3)
    LU, ipiv, info = oracle_mod.getrf(A)
    r, a = oracle_mod.lu_residual_fro(A, LU, ipiv)
    assert r / a <= 10 * n * np.finfo(float).eps
    # the same factors through numpy's independent product
    L, U = oracle_mod.unpack(LU)
    PA = A[oracle_mod.perm_from_ipiv(ipiv, n)]
    assert np.linalg.norm(PA - L @ U) / np.linalg.norm(A) <= 10 * n * np.finfo(float).eps
    # |l_ij| <= 1 is what partial pivoting guarantees
    assert np.max(np.abs(np.tril(LU, -1))) <= 1.0


def test_planted_mistake_is_caught(oracle_mod):
    """A perturbed factor (a plausible dropped term) fails the residual checks."""
    n = 64
    A = li.uniform(n, seed=4)
    LU, ipiv, info = oracle_mod.getrf(A)
    bad = LU.copy()
    bad[40, 12] += 1e-6
    r, a = oracle_mod.lu_residual_fro(A, bad, ipiv)
    assert r / a > 1e-9
    w = li.uniform(n, 1, seed=8)[:, 0]
    rp, ap, wp = oracle_mod.lu_residual_probe(A, bad, ipiv, w)
    assert rp / (ap * wp) > 1e-10
    bad_piv = ipiv.copy()
    bad_piv[[3, 5]] = bad_piv[[5, 3]]
    r2, _ = oracle_mod.lu_residual_fro(A, LU, bad_piv)
    assert r2 / a > 1e-3


def test_probe_matches_direct_residual(oracle_mod):
    n = 150
    A = li.uniform(n, seed=11)
    LU, ipiv, info = oracle_mod.getrf(A)
    w = li.uniform(n, 1, seed=12)[:, 0]
    rp, ap, wp = oracle_mod.lu_residual_probe(A, LU, ipiv, w)
    L, U = oracle_mod.unpack(LU)
    PA = A[oracle_mod.perm_from_ipiv(ipiv, n)]
    direct = np.linalg.norm(PA @ w - L @ (U @ w))
    assert abs(rp - direct) <= 1e-13 * np.linalg.norm(PA @ w)
    assert abs(ap - np.linalg.norm(A)) <= 1e-12 * ap


def test_backward_error_hand_cases(oracle_mod):
    # ||b - Ax|| / (||A|| ||x|| + ||b||): A=[2], x=[1], b=[3] -> 1/(2+3)
    assert oracle_mod.backward_error(np.array([[2.0]]), np.array([1.0]), np.array([3.0])) == pytest.approx(0.2)
    I = np.eye(4)
    b = np.array([1.0, -2.0, 3.0, 0.5])
    assert oracle_mod.backward_error(I, b, b) == 0.0
    # two right-hand sides: the worse one is reported
    A = np.array([[1.0, 0.0], [0.0, 4.0]])
    X = np.array([[1.0, 1.0], [1.0, 0.0]])
    B = np.array([[1.0, 1.0], [4.0, 1.0]])
    # column 1: r = (0, 1), ||A|| = 4, ||x|| = 1, ||b|| = 1 -> 1/5
    assert oracle_mod.backward_error(A, X, B) == pytest.approx(0.2)


def test_getrs_random_matches_numpy(oracle_mod):
    n = 90
    A = li.uniform(n, seed=21)
    B = li.uniform(n, 3, seed=22)
    LU, ipiv, info = oracle_mod.getrf(A)
    X = oracle_mod.getrs(LU, ipiv, B)
    ref = np.linalg.solve(A, B)
    assert np.max(np.abs(X - ref)) / np.max(np.abs(ref)) < 1e-11
    assert oracle_mod.backward_error(A, X, B) < 1e-15


def test_rectangular_tall(oracle_mod):
    A = li.uniform(40, 12, seed=2)
    LU, ipiv, info = oracle_mod.getrf(A)
    assert len(ipiv) == 12
    L = np.tril(LU, -1)[:, :12] + np.eye(40, 12)
    U = np.triu(LU[:12, :])
    PA = A[oracle_mod.perm_from_ipiv(ipiv, 40)]
    assert np.linalg.norm(PA - L @ U) <= 1e-14 * np.linalg.norm(A) * 40


def test_batched_equals_single(oracle_mod):
    sizes = li.batch_sizes(9, 1, 20, seed=3)
    mats = li.batch_matrices(sizes, seed=5)
    rhs = [li.ones_rhs(a) for a in mats]
    LUs, ipivs, infos, xs = oracle_mod.getrf_getrs_batched(mats, rhs)
    for t, A in enumerate(mats):
        LU, ipiv, info = oracle_mod.getrf(A)
        assert np.array_equal(LU, LUs[t]) and np.array_equal(ipiv, ipivs[t])
        assert np.allclose(xs[t], 1.0, atol=1e-10)
        if t % 2 == 1:
            assert np.array_equal(ipiv, np.arange(1, len(ipiv) + 1))


def test_nan_is_never_a_pivot(oracle_mod):
    """Partial pivoting takes the entry of largest magnitude; a NaN has none and
    loses every strict comparison, so it is never chosen, also when it sits on
    the diagonal; a column that is NaN throughout keeps row j."""
    A = np.array([[np.nan, 1.0, 2.0],
                  [0.5, 3.0, 1.0],
                  [-4.0, 1.0, 0.0]])
    LU, piv, info = oracle_mod.getrf(A)
    assert piv[0] == 3                                   # |-4| beats 0.5; the NaN is skipped
    assert np.all(np.isnan(LU[2, :]))                    # the NaN row: NaN multiplier, NaN updates
    assert np.all(np.isfinite(LU[:2, :]))                # the other rows stay finite
    B = np.array([[np.nan, 1.0], [np.nan, 2.0]])
    _, piv2, _ = oracle_mod.getrf(B)
    assert piv2[0] == 1                                  # no candidate: row j itself
    # a NaN below a finite diagonal is skipped as well
    C = np.array([[1.0, 0.0], [np.nan, 1.0]])
    _, piv3, _ = oracle_mod.getrf(C)
    assert piv3[0] == 1


def test_forced_pivot_hand_worked(oracle_mod):
    """The near-tie rule's re-run: a pivot imposed at one step, the others
    searched; hand-worked in tests/golden/lu3x3_forced.txt."""
    g = _read_golden("lu3x3_forced.txt")
    A = np.array([[float(x) for x in r] for r in g["A"]])
    forced = [int(x) for x in g["forced"][0]]
    LU, ipiv, info = oracle_mod.getrf(A, forced=forced)
    assert info == 0
    assert list(ipiv) == [int(x) for x in g["ipiv"][0]]
    L, U = oracle_mod.unpack(LU)
    # every value here is a dyadic rational reached exactly
    assert np.array_equal(L, np.array([[float(x) for x in r] for r in g["L"]]))
    assert np.array_equal(U, np.array([[float(x) for x in r] for r in g["U"]]))
    det = np.prod(np.diag(U)) * (-1) ** int(np.sum(ipiv != np.arange(1, 4)))
    assert det == float(g["det"][0][0])


@pytest.mark.parametrize("seed", range(6))
def test_forced_pivots_match_exact_rational(oracle_mod, seed):
    """Forced choices at random steps (any row at or below the diagonal), the
    rest searched: pivots equal exact rational elimination with the same choices."""
    n = 4 + seed
    h = li.splitmix64(5000 + seed, np.arange(n * n + n, dtype=np.uint64))
    Ai = ((h[:n * n] % np.uint64(2001)).astype(np.int64) - 1000).reshape(n, n)
    forced = [0] * n
    for j in range(0, n - 1, 2):                       # every other step forced
        forced[j] = j + 1 + int(h[n * n + j] % np.uint64(n - j))
    ipiv_x, Lx, Ux = rational_gepp(Ai.tolist(), forced=forced)
    LU, ipiv, info = oracle_mod.getrf(Ai.astype(float), forced=forced)
    assert list(ipiv) == ipiv_x
    L, U = oracle_mod.unpack(LU)
    Lf = np.array([[float(v) for v in r] for r in Lx])
    Uf = np.array([[float(v) for v in r] for r in Ux])
    # forced pivots may give multipliers above 1: bound relative to the exact factors' size
    scale_l = max(1.0, np.max(np.abs(Lf)))
    scale_u = max(1.0, np.max(np.abs(Uf))) * scale_l
    assert np.max(np.abs(L - Lf)) <= 1e-10 * scale_l
    assert np.max(np.abs(U - Uf)) <= 1e-10 * scale_u


def test_forcing_the_searched_pivots_changes_nothing(oracle_mod):
    A = li.uniform(257, seed=31)
    LU, ipiv, info, gaps = oracle_mod.getrf(A, want_gaps=True)
    LUf, ipivf, infof, gapsf = oracle_mod.getrf(A, want_gaps=True, forced=ipiv)
    assert np.array_equal(ipiv, ipivf) and np.array_equal(LU, LUf) and np.array_equal(gaps, gapsf)
    # a forced row above the diagonal is refused
    bad = np.zeros(257, dtype=np.int32)
    bad[5] = 3
    with pytest.raises(ValueError):
        oracle_mod.getrf(A, forced=bad)


# --------------------------------------------------------------------------
# Cholesky (the symmetric positive definite case, A = L L^T)
# --------------------------------------------------------------------------

def _dyadic_spd(n, seed):
    """L lower with diagonal entries in {1, 2, 4} and off-diagonal k/8 (|k| <= 7):
    A = L L^T and every step of the elimination are exact in FP64."""
    h = li.splitmix64(seed, np.arange(n * n + n, dtype=np.uint64))
    k = (h[:n * n] % np.uint64(15)).astype(np.int64).reshape(n, n) - 7
    L = np.tril(k.astype(np.float64) / 8.0, -1)
    L[np.arange(n), np.arange(n)] = 2.0 ** (h[n * n:] % np.uint64(3)).astype(np.float64)
    return L @ L.T, L


def test_cholesky_3x3_hand_worked(oracle_mod):
    g = _read_golden("chol3x3.txt")
    A = np.array([[float(x) for x in r] for r in g["A"]])
    L, info = oracle_mod.potrf(A)
    assert info == 0
    Lx = np.array([[float(x) for x in r] for r in g["L"]])
    assert np.array_equal(np.tril(L), Lx)                 # every value here is exact
    assert np.array_equal(np.triu(L, 1), np.triu(A, 1))   # the upper part is not touched
    assert np.prod(np.diag(L)) ** 2 == float(g["det"][0][0])


@pytest.mark.parametrize("n", [1, 5, 33, 150])
def test_cholesky_dyadic_exact(oracle_mod, n):
    A, L = _dyadic_spd(n, seed=600 + n)
    Lo, info = oracle_mod.potrf(A)
    assert info == 0 and np.array_equal(np.tril(Lo), L)
    # and the solve: x integer, b = A x exact
    x = (li.splitmix64(n, np.arange(n, dtype=np.uint64)) % np.uint64(9)).astype(np.float64) - 4.0
    assert np.array_equal(oracle_mod.potrs(Lo, A @ x), x)


@pytest.mark.parametrize("seed", range(5))
def test_cholesky_brute_force_determinant(oracle_mod, seed):
    n = 3 + seed
    h = li.splitmix64(7000 + seed, np.arange(n * n, dtype=np.uint64))
    M = ((h % np.uint64(11)).astype(np.int64) - 5).reshape(n, n)
    Ai = M @ M.T + n * np.eye(n, dtype=np.int64)             # symmetric positive definite, integer
    L, info = oracle_mod.potrf(Ai.astype(float))
    assert info == 0
    det = float(leibniz_det(Ai.tolist()))
    assert abs(np.prod(np.diag(L)) ** 2 - det) <= 1e-10 * det


def test_cholesky_agrees_with_lu_without_interchanges(oracle_mod):
    """A column diagonally dominant SPD matrix has no interchanges under partial
    pivoting, and then L_chol = L_lu diag(u_jj)^(1/2)."""
    n = 120
    B = li.uniform(n, n, seed=41)
    A = (B + B.T) / 2 + 2 * n * np.eye(n)
    LU, ipiv, info = oracle_mod.getrf(A)
    assert np.array_equal(ipiv, np.arange(1, n + 1))
    Llu, Ulu = oracle_mod.unpack(LU)
    L, info = oracle_mod.potrf(A)
    assert info == 0
    assert np.max(np.abs(np.tril(L) - Llu * np.sqrt(np.diag(Ulu))[None, :])) <= 1e-12 * np.max(np.abs(L))


def test_cholesky_not_positive_definite(oracle_mod):
    L, info = oracle_mod.potrf(np.array([[1.0, 2.0], [2.0, 1.0]]))     # a22 - l21^2 = 1 - 4 < 0
    assert info == 2
    L, info = oracle_mod.potrf(np.array([[0.0, 0.0], [0.0, 1.0]]))
    assert info == 1
