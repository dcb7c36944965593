"""CPU oracle for LU with partial pivoting -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package; the library never imports it and it imports nothing from the
library.  The arithmetic lives in ``lu_oracle.c`` (plain C, FP64,
``-ffp-contract=off``); this module compiles it with gcc and wraps it with
ctypes.  Inputs and outputs are numpy arrays indexed A[i, j].

Functions and the passages they follow:

* ``getrf``   unblocked right-looking LU with partial pivoting (section 3.1,
              Figure 1 left, LU_unb, with the pivoting the same section says
              all codes integrate); pinned by the hand-worked 3x3 case, the
              dyadic P^T L U family, the Wilkinson matrix, Leibniz
              determinants and exact-rational elimination in the tests.
* ``getrs``   P, L and U solves (section 1: LU is the first step of solving
              linear systems); pinned by exact dyadic solves and residuals.
* ``backward_error`` normwise Rigal-Gaches backward error; pinned by
              hand-computed cases.
* ``lu_residual_fro`` / ``lu_residual_probe`` checks of P A = L U.
* ``potrf`` / ``potrs`` unblocked right-looking Cholesky A = L L^T and its
              solves (the symmetric positive definite case section 1 names as
              the next factorization for the same scheme); pinned by a
              hand-worked 3x3 case, exact dyadic factors, the LU of the same
              matrix and a brute-force determinant in the tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lu_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile lu_oracle.c into liboracle.so (gcc, -O2 -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        d, i = ctypes.c_double, ctypes.c_int
        lib.oracle_getrf.argtypes = [i, i, P(d), i, P(i), P(d), i]
        lib.oracle_getrf.restype = i
        lib.oracle_getrf_forced.argtypes = [i, i, P(d), i, P(i), P(d), i, P(i)]
        lib.oracle_getrf_forced.restype = i
        lib.oracle_getrs.argtypes = [i, i, P(d), i, P(i), P(d), i]
        lib.oracle_getrs.restype = i
        lib.oracle_apply_pivots.argtypes = [i, i, P(d), i, P(i), i]
        lib.oracle_lu_residual_fro.argtypes = [i, P(d), i, P(d), i, P(i), P(d)]
        lib.oracle_lu_residual_probe.argtypes = [i, P(d), i, P(d), i, P(i), P(d), P(d)]
        lib.oracle_backward_error.argtypes = [i, i, P(d), i, P(d), i, P(d), i, P(d)]
        lib.oracle_backward_error.restype = d
        lib.oracle_getrf_getrs_batched.argtypes = [i, P(i), P(d), P(ctypes.c_long), P(i),
                                                   P(ctypes.c_long), P(d), P(ctypes.c_long), P(i)]
        lib.oracle_potrf.argtypes = [i, P(d), i]
        lib.oracle_potrf.restype = i
        lib.oracle_potrs.argtypes = [i, i, P(d), i, P(d), i]
        lib.oracle_potrs.restype = i
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _fortran(A):
    return np.asfortranarray(np.asarray(A, dtype=np.float64))


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def getrf(A, nthreads: int = 1, want_gaps: bool = False, forced=None):
    """Return (LU, ipiv, info[, gaps]) for the m x n matrix A (copied).

    ``forced`` (optional, length min(m, n)): 1-based pivot rows imposed on
    the elimination, 0 where the step searches as usual (the near-tie rule:
    re-run with another implementation's choice at a step whose top-2 gap is
    within rounding).  ``gaps`` are always the search's own top-2 gaps."""
    lib = _load()
    F = _fortran(A).copy(order="F")
    m, n = F.shape
    k = min(m, n)
    ipiv = np.zeros(max(k, 1), dtype=np.int32)
    gaps = np.zeros(max(k, 1), dtype=np.float64) if want_gaps else None
    if forced is None:
        info = lib.oracle_getrf(m, n, _dp(F), max(m, 1), _ip(ipiv),
                                _dp(gaps) if want_gaps else None, int(nthreads))
    else:
        fz = np.full(max(k, 1), -1, dtype=np.int32)
        f = np.asarray(forced, dtype=np.int64)[:k]
        fz[:len(f)] = np.where(f > 0, f - 1, -1)
        info = lib.oracle_getrf_forced(m, n, _dp(F), max(m, 1), _ip(ipiv),
                                       _dp(gaps) if want_gaps else None, int(nthreads), _ip(fz))
    if info < 0:
        raise ValueError("oracle_getrf: bad argument")
    out = (F, ipiv[:k], info)
    return out + (gaps[:k],) if want_gaps else out


def getrs(LU, ipiv, B):
    """Solve A X = B given getrf's factors; B is (n,) or (n, nrhs)."""
    lib = _load()
    LU = _fortran(LU)
    n = LU.shape[0]
    vec = np.ndim(B) == 1
    X = _fortran(np.reshape(B, (n, -1))).copy(order="F")
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    lib.oracle_getrs(n, X.shape[1], _dp(LU), max(n, 1), _ip(piv), _dp(X), max(n, 1))
    return X[:, 0].copy() if vec else X


def apply_pivots(X, ipiv):
    """Rows of X interchanged in order by ipiv (returns P X)."""
    lib = _load()
    F = _fortran(np.atleast_2d(X.T).T if np.ndim(X) == 1 else X).copy(order="F")
    if np.ndim(X) == 1:
        F = F.reshape(-1, 1, order="F")
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    lib.oracle_apply_pivots(F.shape[0], F.shape[1], _dp(F), max(F.shape[0], 1), _ip(piv), len(piv))
    return F[:, 0].copy() if np.ndim(X) == 1 else F


def lu_residual_fro(A, LU, ipiv):
    """(||P A - L U||_F, ||A||_F)."""
    lib = _load()
    A = _fortran(A); LU = _fortran(LU)
    out = np.zeros(2)
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    lib.oracle_lu_residual_fro(A.shape[0], _dp(A), A.shape[0], _dp(LU), LU.shape[0], _ip(piv), _dp(out))
    return float(out[0]), float(out[1])


def lu_residual_probe(A, LU, ipiv, w):
    """(||P A w - L U w||_2, ||A||_F, ||w||_2)."""
    lib = _load()
    A = _fortran(A); LU = _fortran(LU)
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(3)
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    lib.oracle_lu_residual_probe(A.shape[0], _dp(A), A.shape[0], _dp(LU), LU.shape[0], _ip(piv),
                                 _dp(w), _dp(out))
    return float(out[0]), float(out[1]), float(out[2])


def backward_error(A, X, B):
    """max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    lib = _load()
    A = _fortran(A)
    n = A.shape[0]
    X = _fortran(np.reshape(X, (n, -1)))
    B = _fortran(np.reshape(B, (n, -1)))
    eta = np.zeros(X.shape[1])
    return float(lib.oracle_backward_error(n, X.shape[1], _dp(A), n, _dp(X), n, _dp(B), n, _dp(eta)))


def getrf_getrs_batched(mats, rhs):
    """Factor and solve each (A_t, b_t); returns (LUs, ipivs, infos, xs)."""
    lib = _load()
    ns = np.array([a.shape[0] for a in mats], dtype=np.int32)
    sq = ns.astype(np.int64) ** 2
    aoff = np.concatenate([[0], np.cumsum(sq)[:-1]]).astype(np.int64)
    voff = np.concatenate([[0], np.cumsum(ns.astype(np.int64))[:-1]]).astype(np.int64)
    Abuf = np.concatenate([_fortran(a).ravel(order="F") for a in mats]) if mats else np.zeros(1)
    Bbuf = np.concatenate([np.asarray(b, dtype=np.float64) for b in rhs]) if mats else np.zeros(1)
    piv = np.zeros(max(int(ns.sum()), 1), dtype=np.int32)
    info = np.zeros(max(len(mats), 1), dtype=np.int32)
    L = ctypes.POINTER(ctypes.c_long)
    lib.oracle_getrf_getrs_batched(len(mats), _ip(ns), _dp(Abuf), aoff.ctypes.data_as(L), _ip(piv),
                                   voff.ctypes.data_as(L), _dp(Bbuf), voff.ctypes.data_as(L), _ip(info))
    LUs, ipivs, xs = [], [], []
    for t, n in enumerate(ns):
        LUs.append(Abuf[aoff[t]:aoff[t] + n * n].reshape(n, n, order="F"))
        ipivs.append(piv[voff[t]:voff[t] + n].copy())
        xs.append(Bbuf[voff[t]:voff[t] + n].copy())
    return LUs, ipivs, info[:len(mats)].copy(), xs


def potrf(A):
    """(L, info) of A = L L^T (lower triangle of A used; L's strictly upper part
    is A's, untouched).  Unblocked right-looking Cholesky."""
    lib = _load()
    F = _fortran(A).copy(order="F")
    n = F.shape[0]
    info = lib.oracle_potrf(n, _dp(F), max(n, 1))
    if info < 0:
        raise ValueError("oracle_potrf: bad argument")
    return F, info


def potrs(L, B):
    """Solve A X = B with the factor of potrf; B is (n,) or (n, nrhs)."""
    lib = _load()
    L = _fortran(L)
    n = L.shape[0]
    vec = np.ndim(B) == 1
    X = _fortran(np.reshape(B, (n, -1))).copy(order="F")
    lib.oracle_potrs(n, X.shape[1], _dp(L), max(n, 1), _dp(X), max(n, 1))
    return X[:, 0].copy() if vec else X


def unpack(LU):
    """(L, U) from the packed {L\\U} storage of a square factor."""
    LU = np.asarray(LU)
    L = np.tril(LU, -1) + np.eye(LU.shape[0])
    U = np.triu(LU)
    return L, U


def perm_from_ipiv(ipiv, m):
    """Row order r such that (P A)[j, :] = A[r[j], :]."""
    r = np.arange(m)
    for j, p in enumerate(np.asarray(ipiv) - 1):
        r[j], r[p] = r[p], r[j]
    return r
