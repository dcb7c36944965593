"""Seeded synthetic inputs for the LU hot path (shared by the CUDA path's tests
and by the oracle's tests; holds none of the factorization's arithmetic).

Every matrix is a pure function of (shape, seed).  Random numbers come from
the counter-based splitmix64 generator (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): the value for counter
``c`` is the finaliser applied to ``seed + (c + 1) * 0x9E3779B97F4A7C15``,
i.e. exactly the (c+1)-th output of a splitmix64 stream started at ``seed``.

The workloads follow the paper's experiments (section 4: square matrices with
random uniform entries) with the interval [-1, 1] used by the benchmark
configurations, plus structured families whose LU factors are known in closed
form (used as pins):

* ``uniform``          A(i,j) = 2 * u(h(seed, j*m + i)) - 1, u = top 53 bits / 2^53
* ``dyadic_plu``       A = P^T L U with L unit-lower, l_ij = k/8 (|k| <= 7) and
                       U upper with small integer entries: partial pivoting
                       recovers P, L and U exactly in any binary precision with
                       at least 24 significand bits.
* ``wilkinson``        a_ii = 1, a_ij = -1 (i > j), a_in = 1: every column step
                       is an all-magnitude tie, growth factor 2^(n-1).
* ``diag_dominant``    uniform plus n on the diagonal: no interchanges.
* ``kappa_matrix``     A = U diag(s) V^T, U and V products of Householder
                       reflectors, s_i = kappa^(-i/(n-1)).
* ``batch_sizes``      order of each member of a batch, uniform integers.

Matrices are returned as numpy arrays indexed A[i, j] (row i, column j).
The helpers ``to_device_colmajor`` / ``from_device_colmajor`` move between that
form and the column-major device layout used by the library (a torch tensor of
shape (n_cols, ld) whose row j holds column j).
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

# Seed recipe for the benchmark workloads: seed = BASE_SEED + 1000*family + case.
BASE_SEED = 20161106


def splitmix64(seed: int, ctr: np.ndarray) -> np.ndarray:
    """splitmix64 output for counters ``ctr`` (uint64 array) of a stream seeded ``seed``."""
    ctr = np.asarray(ctr, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (ctr + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_scalar(seed: int, ctr: int) -> int:
    """Pure-Python splitmix64 (used to pin the vectorised versions)."""
    z = (seed + (ctr + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


def unit_uniform(h: np.ndarray) -> np.ndarray:
    """Top 53 bits of h as a double in [0, 1); exact."""
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(m: int, n: int | None = None, seed: int = 0, lo: float = -1.0) -> np.ndarray:
    """m x n matrix with A(i,j) = lo + (1-lo) * u(h(seed, j*m + i)).

    With lo = -1 the entries are iid uniform on [-1, 1) and exact in FP64
    (2u - 1 needs at most 53 bits).  lo = 0 gives the paper's (0, 1) variant.
    """
    n = m if n is None else n
    # counter j*m + i -> column-major fill, generated a block of columns at a
    # time to bound the temporaries; large matrices come back Fortran-ordered
    # (same values, no transposing copy)
    out = np.empty((n, m), dtype=np.float64)
    cols = max(1, (1 << 24) // max(m, 1))
    for j0 in range(0, n, cols):
        j1 = min(n, j0 + cols)
        c = np.arange(j0 * m, j1 * m, dtype=np.uint64)
        u = unit_uniform(splitmix64(seed, c))
        v = lo + (1.0 - lo) * u if lo != -1.0 else 2.0 * u - 1.0
        out[j0:j1] = v.reshape(j1 - j0, m)
    return out.T.copy() if m * n <= (1 << 24) else out.T


def uniform_colmajor_torch(m: int, n: int, seed: int, device, dtype=None, ld: int | None = None):
    """Same values as ``uniform(m, n, seed)`` built directly in the device
    column-major layout (torch tensor of shape (n, ld), row j = column j).

    Uses int64 arithmetic (two's complement wrap-around equals uint64 mod 2^64)
    and masked shifts to emulate logical shifts.
    """
    import torch

    ld = m if ld is None else ld
    dtype = torch.float64 if dtype is None else dtype
    out = torch.zeros((n, ld), dtype=dtype, device=device)
    # generate column blocks to bound temporary memory
    cols_per_chunk = max(1, (1 << 26) // max(m, 1))
    for j0 in range(0, n, cols_per_chunk):
        j1 = min(n, j0 + cols_per_chunk)
        c = torch.arange(j0 * m, j1 * m, dtype=torch.int64, device=device)
        h = _splitmix64_torch(seed, c)
        u = ((h >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
        v = 2.0 * u - 1.0
        out[j0:j1, :m] = v.view(j1 - j0, m).to(dtype)
    return out


def _s64(x: int) -> int:
    x &= MASK64
    return x - (1 << 64) if x >> 63 else x


def _splitmix64_torch(seed: int, c):
    import torch

    g = _s64(GAMMA)
    z = (c + 1) * g + _s64(seed)
    z = (z ^ ((z >> 30) & ((1 << 34) - 1))) * _s64(M1)
    z = (z ^ ((z >> 27) & ((1 << 37) - 1))) * _s64(M2)
    z = z ^ ((z >> 31) & ((1 << 33) - 1))
    return z


def ones_rhs(A: np.ndarray) -> np.ndarray:
    """b = A * ones(n), summed left to right in FP64 (fixed order)."""
    b = np.zeros(A.shape[0])
    for j in range(A.shape[1]):
        b += A[:, j]
    return b


def permutation(n: int, seed: int) -> np.ndarray:
    """Seeded permutation of 0..n-1 (Fisher-Yates driven by splitmix64)."""
    p = np.arange(n)
    if n <= 1:
        return p
    h = splitmix64(seed, np.arange(n, dtype=np.uint64))
    for i in range(n - 1, 0, -1):
        r = int(h[i] % np.uint64(i + 1))
        p[i], p[r] = p[r], p[i]
    return p


def dyadic_factors(n: int, seed: int):
    """(perm, L, U) with L unit-lower, l_ij = k/8 for k in [-7, 7] (i > j),
    U upper with integer entries in [-8, 8] and a nonzero diagonal.

    ``perm[r]`` is the row of P^T L U that holds row r of L U, i.e.
    A[perm[r], :] = (L U)[r, :].
    """
    hl = splitmix64(seed, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    hu = splitmix64(seed ^ 0x5A5A5A5A, np.arange(n * n, dtype=np.uint64)).reshape(n, n)
    k = (hl % np.uint64(15)).astype(np.int64) - 7
    L = np.tril(k.astype(np.float64) / 8.0, -1) + np.eye(n)
    ui = (hu % np.uint64(17)).astype(np.int64) - 8
    U = np.triu(ui.astype(np.float64))
    d = np.diag(U).copy()
    d[d == 0] = 1.0
    np.fill_diagonal(U, d)
    perm = permutation(n, seed ^ 0x33CC33CC)
    return perm, L, U


def dyadic_plu(n: int, seed: int):
    """A = P^T L U built from ``dyadic_factors``; every entry and every partial
    sum is a multiple of 1/8 bounded by 8*7*n, so the product is exact in FP64."""
    perm, L, U = dyadic_factors(n, seed)
    LU = L @ U
    A = np.empty_like(LU)
    A[perm, :] = LU
    return A, perm, L, U


def wilkinson(n: int) -> np.ndarray:
    """Wilkinson's growth matrix: 1 on the diagonal and in the last column, -1 below the diagonal."""
    A = np.tril(-np.ones((n, n)), -1) + np.eye(n)
    A[:, n - 1] = 1.0
    return A


def diag_dominant(n: int, seed: int) -> np.ndarray:
    """uniform(n, seed) with n added to the diagonal (strictly column diagonally dominant)."""
    A = uniform(n, n, seed)
    A[np.arange(n), np.arange(n)] += n
    return A


def kappa_singular_values(n: int, kappa: float) -> np.ndarray:
    """s_i = kappa^(-i/(n-1)), i = 0..n-1 (geometric from 1 down to 1/kappa)."""
    if n == 1:
        return np.ones(1)
    i = np.arange(n, dtype=np.float64)
    return np.power(float(kappa), -i / (n - 1))


def householder_vectors(n: int, k: int, seed: int) -> np.ndarray:
    """n x k matrix whose columns are the reflector vectors v ~ U[-1, 1)."""
    return uniform(n, k, seed)


def apply_reflectors(V: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Return H_1 H_2 ... H_k X with H_t = I - 2 v_t v_t^T / (v_t^T v_t)."""
    X = X.copy()
    for t in range(V.shape[1] - 1, -1, -1):
        v = V[:, t]
        X -= np.outer(v, (2.0 / (v @ v)) * (v @ X))
    return X


def kappa_matrix(n: int, kappa: float, seed: int, k: int | None = None) -> np.ndarray:
    """A = U diag(s) V^T with U = H_1..H_k (seeded), V likewise, s geometric.

    k reflectors per side (default n).  Dense numpy: for moderate n only; the
    device builder ``kappa_matrix_torch`` computes the same product."""
    k = n if k is None else k
    s = kappa_singular_values(n, kappa)
    Vu = householder_vectors(n, k, seed)
    Vv = householder_vectors(n, k, seed + 1)
    X = apply_reflectors(Vv, np.eye(n)).T  # V^T
    X = s[:, None] * X
    return apply_reflectors(Vu, X)


def kappa_matrix_torch(n: int, kappa: float, seed: int, k: int, device, block: int = 64):
    """Device builder of ``kappa_matrix`` (FP64, column-major (n, n) tensor whose
    row j is column j of A).  Reflectors are applied in blocks of ``block`` with
    the compact WY form H_1..H_b = I - Y T Y^T (Schreiber and Van Loan, 1989),
    using library matrix products; it is input construction only."""
    import torch

    s = torch.from_numpy(kappa_singular_values(n, kappa)).to(device)
    Q_u, Vt = kappa_factors_torch(n, seed, k, device, block)
    A = Q_u @ (s[:, None] * Vt)
    return A.T.contiguous()  # row j = column j


def kappa_from_factors_torch(Q_u, Vt, kappa: float):
    """A = U diag(s) V^T for the factors of ``kappa_factors_torch`` (one library
    product per kappa), in the device column-major layout."""
    import torch

    n = Q_u.shape[0]
    s = torch.from_numpy(kappa_singular_values(n, kappa)).to(Q_u.device)
    return (Q_u @ (s[:, None] * Vt)).T.contiguous()


def kappa_factors_torch(n: int, seed: int, k: int, device, block: int = 64):
    """(U, V^T) of ``kappa_matrix``: U = H_1..H_k from the reflectors of
    ``seed``, V likewise from ``seed + 1``, both explicit FP64 n x n (row-major
    torch tensors).  Shared by every kappa of one (order, seed)."""
    import torch

    Vu = torch.from_numpy(householder_vectors(n, k, seed)).to(device)
    Vv = torch.from_numpy(householder_vectors(n, k, seed + 1)).to(device)

    def wy(Y):
        b = Y.shape[1]
        tau = 2.0 / (Y * Y).sum(0)
        T = torch.zeros(b, b, dtype=torch.float64, device=device)
        for t in range(b):
            T[t, t] = tau[t]
            if t:
                T[:t, t] = -tau[t] * (T[:t, :t] @ (Y[:, :t].T @ Y[:, t]))
        return T

    def apply_left(Vs, X):
        # X <- H_1 ... H_k X, processed from the last block to the first
        for b0 in range(((Vs.shape[1] - 1) // block) * block, -1, -block):
            Y = Vs[:, b0:b0 + block]
            T = wy(Y)
            X -= Y @ (T @ (Y.T @ X))
        return X

    Vt = apply_left(Vv, torch.eye(n, dtype=torch.float64, device=device)).T.contiguous()
    del Vv
    Q_u = apply_left(Vu, torch.eye(n, dtype=torch.float64, device=device))
    return Q_u, Vt


def batch_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """count integers uniform on [lo, hi] (inclusive)."""
    h = splitmix64(seed, np.arange(count, dtype=np.uint64))
    return (lo + (h % np.uint64(hi - lo + 1)).astype(np.int64)).astype(np.int64)


def batch_matrices(sizes, seed: int):
    """Batch of uniform matrices; odd members get n_i added to the diagonal."""
    out = []
    for i, n in enumerate(sizes):
        A = uniform(int(n), int(n), seed + 7919 * i)
        if i % 2 == 1:
            A[np.arange(n), np.arange(n)] += n
        out.append(A)
    return out


def to_device_colmajor(A: np.ndarray, device, dtype=None, ld: int | None = None):
    """numpy A[i, j] (m x n) -> torch (n, ld) tensor whose row j holds column j."""
    import torch

    m, n = A.shape
    ld = m if ld is None else ld
    dtype = torch.float64 if dtype is None else dtype
    t = torch.zeros((n, ld), dtype=dtype)
    t[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T)).to(dtype)
    return t.to(device)


def from_device_colmajor(t, m: int | None = None) -> np.ndarray:
    """Inverse of ``to_device_colmajor`` (returns float64 numpy A[i, j])."""
    import torch

    n, ld = t.shape
    m = ld if m is None else m
    return t[:, :m].to(torch.float64).cpu().numpy().T.copy()
