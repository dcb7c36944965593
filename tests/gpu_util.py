"""Helpers for the GPU parity tests (device buffers from seeded inputs)."""
import numpy as np

import lu_inputs as li

EPS64 = np.finfo(np.float64).eps
EPS32 = float(np.finfo(np.float32).eps)


def dev():
    import torch
    return torch.device("cuda:0")


def factor_gpu(A, dtype="f64", ld=None, **opts):
    """Run lu_factor on A (numpy, row-major indexing); returns (LU numpy f64, ipiv, info)."""
    import torch

    import paper_1611_06365_gb300 as lu

    n = A.shape[0]
    tdt = torch.float64 if dtype == "f64" else torch.float32
    dA = li.to_device_colmajor(A, dev(), dtype=tdt, ld=ld)
    ipiv = torch.zeros(max(n, 1), dtype=torch.int32, device=dev())
    info = torch.full((1,), -7, dtype=torch.int32, device=dev())
    lu.lu_factor(dA, ipiv, info, n, **opts)
    torch.cuda.synchronize()
    return li.from_device_colmajor(dA, n), ipiv.cpu().numpy()[:n], int(info.item()), dA, ipiv


def expected_ipiv(perm):
    n = len(perm)
    cur = list(range(n))
    where = list(range(n))
    out = []
    for j in range(n):
        p = where[perm[j]]
        out.append(p + 1)
        rj, rp = cur[j], cur[p]
        cur[j], cur[p] = rp, rj
        where[rp], where[rj] = j, p
    return np.array(out, dtype=np.int32)
