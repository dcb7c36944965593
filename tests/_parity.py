"""Full-vector pivot parity with the oracle, with the near-tie rule.

The FP64 GPU path and the oracle perform the same partial-pivoting
elimination (section 3.1) but round differently (fused multiply-adds and a
blocked summation order on the GPU, two roundings per update in the oracle).
Their pivot vectors must agree entry for entry.  The one allowed exception is
a step j where the oracle's two largest candidates are closer than rounding
can resolve: top-2 relative gap g_j <= 64 n eps.  There the GPU's choice is
equally valid; the oracle is re-run with that pivot forced at step j
(``oracle.getrf(..., forced=...)``) and the comparison continues from the
re-run.  A mismatch at a step with a larger gap fails.
"""
from __future__ import annotations

import numpy as np

EPS64 = np.finfo(np.float64).eps


EPS32 = float(np.finfo(np.float32).eps)


def tie_bound(n: int, eps: float = EPS64) -> float:
    return 64.0 * n * eps


def oracle_parity(oracle_mod, A, ipiv_gpu, max_reruns: int = 4, threads: int | None = None, eps: float = EPS64):
    """Compare the GPU's pivots with the oracle's under the near-tie rule.

    eps: the unit roundoff of the GPU's arithmetic (FP64 by default; an FP32
    factorization is compared with the oracle run on its FP32-rounded input,
    where rounding can reorder candidates up to 64 n eps32 apart).
    Returns (LU of the final oracle run, list of (step, gap) re-runs).  Raises
    AssertionError at a mismatch whose gap exceeds the bound, or after
    max_reruns forced re-runs."""
    n = A.shape[0]
    bound = tie_bound(n, eps)
    threads = oracle_mod.default_threads() if threads is None else threads
    ipiv_gpu = np.asarray(ipiv_gpu, dtype=np.int32)
    forced = np.zeros(n, dtype=np.int32)
    LUo, pivo, info, gaps = oracle_mod.getrf(A, nthreads=threads, want_gaps=True)
    reruns = []
    while True:
        bad = np.nonzero(ipiv_gpu[:len(pivo)] != pivo)[0]
        if bad.size == 0:
            return LUo, reruns
        j = int(bad[0])
        assert gaps[j] <= bound, (
            f"pivot mismatch at step {j}: GPU row {ipiv_gpu[j]}, oracle row {pivo[j]}, "
            f"top-2 gap {gaps[j]:.3e} > {bound:.3e}")
        assert len(reruns) < max_reruns, f"more than {max_reruns} near-tie re-runs: {reruns}"
        reruns.append((j, float(gaps[j])))
        forced[j] = ipiv_gpu[j]
        LUo, pivo, info, gaps = oracle_mod.getrf(A, nthreads=threads, want_gaps=True, forced=forced)


def golden_agreement(ipiv_gpu, ipiv_golden, near: dict, n: int):
    """Agreement with a stored oracle pivot vector (no re-run possible).

    Returns {"pivot_agreement": fraction of equal entries, "first_mismatch_step":
    j or None, "first_mismatch_gap": gap or None, "tie_ambiguous": bool}; a first
    mismatch is tie-ambiguous when the stored gap of that step is within the bound
    (steps without a stored gap had gaps >= 1e-6, far above it)."""
    g = np.asarray(ipiv_gpu, dtype=np.int32)
    o = np.asarray(ipiv_golden, dtype=np.int32)
    eq = g == o
    out = {"pivot_agreement": float(eq.mean()), "first_mismatch_step": None, "first_mismatch_gap": None,
           "tie_ambiguous": False}
    if not eq.all():
        j = int(np.argmin(eq))
        gap = near.get(j)
        out.update(first_mismatch_step=j, first_mismatch_gap=gap,
                   tie_ambiguous=gap is not None and gap <= tie_bound(n))
    return out
