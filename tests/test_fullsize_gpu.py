"""Checks at the configurations' full sizes, in the launch configuration the
benchmark times (default options): outputs the oracle can compute exactly on
a sample (the first panel's pivots and factors depend only on the first
columns of A), and properties that hold at any size (multipliers |l| <= 1 of
partial pivoting, a randomized residual probe of P A = L U, the backward
error of the solve), for the FP64 order sweep, the mixed-precision solve and
the whole 10 000-matrix batch."""
import numpy as np
import pytest

import lu_inputs as li
from tests.gpu_util import EPS64, dev

pytestmark = pytest.mark.gpu

FAMILY_SEED = 20161106          # seed = FAMILY_SEED + 1000 * configuration + case


def _host_f(t, n):
    """Device column-major (n, ld) tensor -> Fortran-ordered numpy n x n view."""
    return t[:, :n].cpu().numpy().T


def _first_panel_matches(oracle_mod, A_f, LU_f, ipiv, k, n):
    """The first k pivots and columns of L (and U's leading k x k block) agree with
    the oracle's unblocked elimination of A[:, :k]; a pivot differing where the
    oracle's top-2 gap is below 64 n eps is a rounding tie, after which the rest
    cannot be compared."""
    LUo, pivo, info, gaps = oracle_mod.getrf(np.asfortranarray(A_f[:, :k]), nthreads=oracle_mod.default_threads(),
                                              want_gaps=True)
    assert info == 0
    for j in range(k):
        if ipiv[j] != pivo[j]:
            assert gaps[j] <= 64 * n * EPS64, (j, ipiv[j], pivo[j], gaps[j])
            return
    # the later panels' interchanges also move the rows of these L columns
    later = np.concatenate([np.arange(1, k + 1, dtype=np.int32), ipiv[k:]])
    LUo = oracle_mod.apply_pivots(LUo, later)
    scale = max(1.0, float(np.max(np.abs(LUo))))
    assert np.max(np.abs(LU_f[:, :k] - LUo)) <= 100 * k * EPS64 * scale


@pytest.mark.parametrize("n,case", [(4096, 1), (8192, 2), (16384, 0), (32768, 3)])
def test_fp64_full_size(oracle_mod, n, case):
    import torch

    import paper_1611_06365_gb300 as lu
    seed = FAMILY_SEED + 1000 * 2 + case
    A = li.uniform_colmajor_torch(n, n, seed, dev(), torch.float64)
    dA = A.clone()
    ipiv = torch.zeros(n, dtype=torch.int32, device=dev())
    info = torch.full((1,), -1, dtype=torch.int32, device=dev())
    lu.lu_factor(dA, ipiv, info, n)
    b = (A.t() @ torch.ones(n, dtype=torch.float64, device=dev())).view(1, n)
    x = b.clone()
    lu.lu_solve(dA, ipiv, x, n)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    # partial pivoting: every multiplier has magnitude <= 1 (column j of L is row j of dA, past the diagonal)
    assert float(torch.triu(dA, diagonal=1).abs().max()) <= 1.0
    A_f, LU_f = _host_f(A, n), _host_f(dA, n)
    piv = ipiv.cpu().numpy()
    del dA
    _first_panel_matches(oracle_mod, A_f, LU_f, piv, 64, n)
    rng = np.random.default_rng(seed)
    for _ in range(2):
        w = rng.standard_normal(n)
        r, a, wn = oracle_mod.lu_residual_probe(A_f, LU_f, piv, w)
        assert r / (a * wn) <= 10 * n * EPS64
    xh = x.view(-1).cpu().numpy()
    bh = b.view(-1).cpu().numpy()
    assert oracle_mod.backward_error(A_f, xh, bh) <= 10 * n * EPS64
    assert np.max(np.abs(xh - 1.0)) <= 1e-6


@pytest.mark.parametrize("n,kappa,nrhs,case,rung_max", [
    (16384, 1e2, 1, 0, 0),
    (16384, 1e5, 8, 1, 1),
    (16384, 1e8, 1, 2, 2),
    (32768, 1e5, 1, 3, 1),
])
def test_mixed_full_size(oracle_mod, n, kappa, nrhs, case, rung_max):
    import torch

    import paper_1611_06365_gb300 as lu
    seed = FAMILY_SEED + 1000 * 3 + case
    A = li.kappa_matrix_torch(n, kappa, seed, 256, dev())
    Xt = torch.from_numpy(li.uniform(n, nrhs, seed + 1)).to(dev())
    Xt[:, 0] = 1.0
    Xt = Xt.t().contiguous()                      # (nrhs, n): row q = right-hand side q
    B = (A.t() @ Xt.t()).t().contiguous()         # B = A X_true in FP64
    X = torch.zeros_like(B)
    rep = lu.lu_solve_mixed(A, B, X, n)
    torch.cuda.synchronize()
    A_f = _host_f(A, n)
    Xh = X.cpu().numpy().T
    eta = oracle_mod.backward_error(A_f, Xh, B.cpu().numpy().T)
    assert eta <= 1e-14 and rep.backward_error <= 1e-14, (rep.as_dict(), eta)
    assert rep.rung <= rung_max
    fwd = np.max(np.abs(Xh - Xt.cpu().numpy().T)) / np.max(np.abs(Xt.cpu().numpy()))
    assert fwd <= 100 * kappa * max(eta, 1e-16)


def _batch(dtype):
    import torch
    sizes = li.batch_sizes(10000, 16, 256, seed=FAMILY_SEED + 1000 * 4)
    mats = li.batch_matrices(sizes, seed=FAMILY_SEED + 1000 * 4 + 1)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    offs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 2)])
    roffs = np.concatenate([[0], np.cumsum(sizes.astype(np.int64))])
    flat = np.concatenate([np.asfortranarray(a).ravel(order="F") for a in mats])
    buf = torch.from_numpy(flat).to(dev(), tdt)
    rhs = torch.from_numpy(np.concatenate([li.ones_rhs(a) for a in mats])).to(dev(), tdt)
    esz = buf.element_size()
    ns = torch.tensor(sizes, dtype=torch.int32, device=dev())
    ptrA = torch.tensor([buf.data_ptr() + int(o) * esz for o in offs[:-1]], dtype=torch.int64, device=dev())
    ipiv = torch.zeros(int(roffs[-1]), dtype=torch.int32, device=dev())
    ptrP = torch.tensor([ipiv.data_ptr() + int(o) * 4 for o in roffs[:-1]], dtype=torch.int64, device=dev())
    ptrB = torch.tensor([rhs.data_ptr() + int(o) * esz for o in roffs[:-1]], dtype=torch.int64, device=dev())
    info = torch.zeros(10000, dtype=torch.int32, device=dev())
    return sizes, mats, offs, roffs, buf, rhs, ns, ptrA, ipiv, ptrP, ptrB, info


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_full_10000(oracle_mod, dtype):
    """The whole batch in one factorization launch and one solve launch: FP64
    pivots equal the oracle's for every member (up to rounding ties), the
    diagonally dominant half has no interchanges, and every solution has a small
    backward error in its precision."""
    import torch

    import paper_1611_06365_gb300 as lu
    sizes, mats, offs, roffs, buf, rhs, ns, ptrA, ipiv, ptrP, ptrB, info = _batch(dtype)
    code = lu.LU_F64 if dtype == "f64" else lu.LU_F32
    lu.lu_factor_batched(code, ns, ptrA, ns, ptrP, info, 256)
    lu.lu_solve_batched(code, 1, ns, ptrA, ns, ptrP, ptrB, ns, 256)
    torch.cuda.synchronize()
    assert int((info != 0).sum()) == 0
    piv = ipiv.cpu().numpy()
    x = rhs.cpu().numpy().astype(np.float64)
    eps = EPS64 if dtype == "f64" else float(np.finfo(np.float32).eps)
    if dtype == "f64":
        _, pivs_o, infos_o, _ = oracle_mod.getrf_getrs_batched(mats, [li.ones_rhs(a) for a in mats])
        assert np.all(infos_o == 0)
    for t, A in enumerate(mats):
        n = A.shape[0]
        p = piv[roffs[t]:roffs[t + 1]]
        if t % 2 == 1:
            assert np.array_equal(p, np.arange(1, n + 1)), t
        if dtype == "f64":
            if not np.array_equal(p, pivs_o[t]):
                _, _, _, gaps = oracle_mod.getrf(A, want_gaps=True)
                j = int(np.argmax(p != pivs_o[t]))
                assert gaps[j] <= 64 * n * eps, (t, j)
        Ar = A.astype(np.float32).astype(np.float64) if dtype == "f32" else A
        xt = x[roffs[t]:roffs[t + 1]]
        b = li.ones_rhs(A)
        r = np.max(np.abs(b - Ar @ xt))
        eta = r / (np.max(np.sum(np.abs(Ar), axis=1)) * np.max(np.abs(xt)) + np.max(np.abs(b)))
        assert eta <= 10 * n * eps + (2 * eps if dtype == "f32" else 0.0), (t, eta)
