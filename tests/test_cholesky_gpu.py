"""Cholesky factorization on the look-ahead schedule (lu_cholesky) against the
oracle (unblocked right-looking Cholesky, FP64): exact recovery of dyadic
factors on every path, entries within 10 n eps of the oracle's, the residual
of A = L L^T, the solve, the not-positive-definite info, the untouched upper
triangle, and bit-identity across schedules."""
import numpy as np
import pytest

import lu_inputs as li
from tests.gpu_util import EPS32, EPS64, dev

pytestmark = pytest.mark.gpu


def _dyadic_spd(n, seed):
    h = li.splitmix64(seed, np.arange(n * n + n, dtype=np.uint64))
    k = (h[:n * n] % np.uint64(15)).astype(np.int64).reshape(n, n) - 7
    L = np.tril(k.astype(np.float64) / 8.0, -1)
    L[np.arange(n), np.arange(n)] = 2.0 ** (h[n * n:] % np.uint64(3)).astype(np.float64)
    return L @ L.T, L


def _spd(n, seed):
    B = li.uniform(n, n, seed)
    return (B + B.T) / 2 + n * np.eye(n)


def _chol_gpu(A, dtype="f64", ld=None, **opts):
    import torch

    import paper_1611_06365_gb300 as lu
    n = A.shape[0]
    tdt = torch.float64 if dtype == "f64" else torch.float32
    dA = li.to_device_colmajor(A, dev(), dtype=tdt, ld=ld)
    info = torch.full((1,), -7, dtype=torch.int32, device=dev())
    lu.lu_cholesky(dA, info, n, **opts)
    torch.cuda.synchronize()
    return li.from_device_colmajor(dA, n), int(info.item()), dA


@pytest.mark.parametrize("dtype,update", [("f64", 0), ("f64", 4), ("f32", 0)])
@pytest.mark.parametrize("n", [40, 300, 1030])
def test_cholesky_dyadic_exact(n, dtype, update):
    A, L = _dyadic_spd(n, seed=700 + n)
    got, info, _ = _chol_gpu(A, dtype, update=update)
    assert info == 0
    assert np.array_equal(np.tril(got), L)
    assert np.array_equal(np.triu(got, 1), np.triu(A, 1))    # the strictly upper part is not touched


@pytest.mark.parametrize("update", [0, 4])
@pytest.mark.parametrize("n", [1, 63, 64, 65, 500, 1537])
def test_cholesky_matches_oracle(oracle_mod, n, update):
    A = _spd(n, seed=800 + n)
    got, info, _ = _chol_gpu(A, "f64", update=update)
    Lo, info_o = oracle_mod.potrf(A)
    assert info == info_o == 0
    L, Lo = np.tril(got), np.tril(Lo)
    assert np.max(np.abs(L - Lo)) <= 10 * n * EPS64 * np.max(np.abs(Lo))
    assert np.linalg.norm(A - L @ L.T) / np.linalg.norm(A) <= 10 * n * EPS64


def test_cholesky_f32(oracle_mod):
    n = 700
    A = _spd(n, seed=17)
    got, info, _ = _chol_gpu(A, "f32")
    Lo, _ = oracle_mod.potrf(A.astype(np.float32).astype(np.float64))
    assert info == 0
    assert np.max(np.abs(np.tril(got) - np.tril(Lo))) <= 10 * n * EPS32 * np.max(np.abs(Lo))


def test_cholesky_solve(oracle_mod):
    import torch

    import paper_1611_06365_gb300 as lu
    n, nrhs = 900, 3
    A = _spd(n, seed=21)
    got, info, dA = _chol_gpu(A, "f64", update=4)
    B = li.uniform(n, nrhs, seed=22)
    dB = li.to_device_colmajor(B, dev())
    lu.lu_cholesky_solve(dA, dB, n)
    torch.cuda.synchronize()
    X = li.from_device_colmajor(dB, n)
    assert oracle_mod.backward_error(A, X, B) <= 10 * n * EPS64
    Xo = oracle_mod.potrs(oracle_mod.potrf(A)[0], B)
    assert np.max(np.abs(X - Xo)) <= 1e3 * n * EPS64 * np.max(np.abs(Xo))


def test_cholesky_not_positive_definite(oracle_mod):
    n = 300
    A = _spd(n, seed=31)
    A[150, 150] = -1.0                      # the updated diagonal of column 151 goes negative
    got, info, _ = _chol_gpu(A, "f64")
    _, info_o = oracle_mod.potrf(A)
    assert info == info_o > 0


def test_cholesky_schedule_invariance_and_padding():
    A = _spd(777, seed=41)
    ref, _, _ = _chol_gpu(A, "f64", nb=48, lookahead=-1)
    for la in (0, 1):
        got, _, _ = _chol_gpu(A, "f64", nb=48, lookahead=la)
        assert np.array_equal(np.tril(got), np.tril(ref))
    emu_ref, _, _ = _chol_gpu(A, "f64", update=4, lookahead=-1)
    emu, _, dA = _chol_gpu(A, "f64", update=4, ld=790)
    assert np.array_equal(np.tril(emu), np.tril(emu_ref))
    assert float(dA[:, 777:].abs().sum()) == 0.0           # padding rows untouched


@pytest.mark.parametrize("update", [0, 4])
def test_cholesky_full_size_8192(update):
    """n = 8192: randomized residual probe of A = L L^T in FP64."""
    import torch

    import paper_1611_06365_gb300 as lu
    n = 8192
    B = li.uniform_colmajor_torch(n, n, 20161106 + 9000, dev(), torch.float64)
    A = (B + B.t()) / 2 + n * torch.eye(n, dtype=torch.float64, device=dev())
    dA = A.clone()
    info = torch.full((1,), -1, dtype=torch.int32, device=dev())
    lu.lu_cholesky(dA, info, n, update=update)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    L = torch.tril(dA.t())                   # row-major view of the column-major factor
    rng = np.random.default_rng(5)
    for _ in range(2):
        w = torch.from_numpy(rng.standard_normal(n)).to(dev())
        r = A.t() @ w - L @ (L.t() @ w)      # A is symmetric: A.t() holds A
        assert float(r.norm() / (A.norm() * w.norm())) <= 10 * n * EPS64
