"""Write the oracle's pivot vectors for the large uniform LU workloads.

The full oracle (plain unblocked GEPP of section 3.1, Figure 1 left, with the
partial pivoting that section says every code integrates) takes minutes at
order 16384 and about an hour at 32768 on a few host cores, too long to run
inside a test or a benchmark.  This script runs it once per (order, seed) and
stores what the GPU parity checks compare against:

  oracle_ipiv_n<order>_s<seed>.txt.gz
    '#' header lines (order, seed, generator, oracle build, wall time);
    'near <j> <gap>' for every step j whose top-2 relative gap
        (|p1| - |p2|) / |p1| is below 1e-6 (the near-tie rule needs the gap
        only where a rounding difference could flip the choice);
    then one 1-based pivot per line, LAPACK sequential-interchange meaning.

It imports only the oracle and the seeded generators.  Usage:

  python tests/golden/make_oracle_pivots.py 16384:20163106 32768:20163109 [--threads T]
"""
from __future__ import annotations

import argparse
import gzip
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

NEAR_GAP = 1e-6


def golden_path(n: int, seed: int) -> str:
    return os.path.join(HERE, f"oracle_ipiv_n{n}_s{seed}.txt.gz")


def write(n: int, seed: int, threads: int) -> str:
    import lu_inputs as li
    import oracle

    A = li.uniform(n, n, seed)
    t0 = time.time()
    _, ipiv, info, gaps = oracle.getrf(A, nthreads=threads, want_gaps=True)
    wall = time.time() - t0
    del A
    path = golden_path(n, seed)
    tmp = path + ".tmp"
    with gzip.open(tmp, "wt") as f:
        f.write(f"# oracle getrf pivots (unblocked GEPP, FP64, -ffp-contract=off), order {n}\n")
        f.write(f"# matrix: lu_inputs.uniform({n}, {n}, seed={seed}), entries uniform [-1, 1)\n")
        f.write(f"# info {info}; {threads} threads; {wall:.0f} s\n")
        for j in np.nonzero(gaps < NEAR_GAP)[0]:
            f.write(f"near {int(j)} {float(gaps[j]):.6e}\n")
        for p in ipiv:
            f.write(f"{int(p)}\n")
    os.replace(tmp, path)
    return path


def read(n: int, seed: int):
    """(ipiv int32 array, {step: gap} for the near ties) or None if absent."""
    path = golden_path(n, seed)
    if not os.path.exists(path):
        return None
    piv, near = [], {}
    with gzip.open(path, "rt") as f:
        for line in f:
            if line.startswith("#"):
                continue
            if line.startswith("near"):
                _, j, g = line.split()
                near[int(j)] = float(g)
            else:
                piv.append(int(line))
    arr = np.array(piv, dtype=np.int32)
    if arr.shape != (n,):
        raise ValueError(f"{path}: {arr.shape[0]} pivots, expected {n}")
    return arr, near


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("cases", nargs="+", help="order:seed pairs")
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    import oracle

    threads = args.threads or oracle.default_threads()
    for c in args.cases:
        n, seed = (int(x) for x in c.split(":"))
        print(write(n, seed, threads), flush=True)


if __name__ == "__main__":
    main()
