"""Write the oracle's eigenvalues for a fixed subset of the mixed-precision workload
(n = 2000, 4x4x4 k-points, one spin, seed 4: ``synth.scaled_cell(2000, seed=4,
kgrid=(4, 4, 4), nspin=1, ill_conditioned=False)``) to ``mixed_n2000_oracle_eps.txt``.

Only the seeded input generator and ``oracle/`` run here (Parts 1-4 of Sec. 3: Bloch sums,
Eigen_HH of S, the cutoff, X^H H X, Eigen_HH of H').  The benchmark and the GPU tests read the
file to state the mixed-precision path's eigenvalue error against the oracle, before and after
its refinement sweep, without running the oracle for minutes each time.

    python tests/golden/make_mixed_n2000_oracle.py        # ~5 min on 8 cores
"""
import os
import sys
from concurrent.futures import ProcessPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

PROBLEMS = (0, 21)   # k-point indices of the 4x4x4 grid (one spin: problem = k)
OUT = os.path.join(HERE, "mixed_n2000_oracle_eps.txt")


def _cell():
    from paper_1402_4247_gb300 import synth
    return synth.scaled_cell(2000, seed=4, kgrid=(4, 4, 4), nspin=1, ill_conditioned=False)


def _solve(p):
    import oracle
    inp = _cell()
    Hk = oracle.bloch_sum(inp.HR[0], inp.R, inp.kpts[p:p + 1])[0]
    Sk = oracle.bloch_sum(inp.SR, inp.R, inp.kpts[p:p + 1])[0]
    eps, C, m, s = oracle.generalized_eigensolve(Hk, Sk)
    return p, m, eps


def main():
    with ProcessPoolExecutor(max_workers=len(PROBLEMS)) as ex:
        res = list(ex.map(_solve, PROBLEMS))
    with open(OUT, "w") as fh:
        fh.write("# Oracle eigenvalues (Ha) of the mixed-precision workload: n = 2000, 4x4x4 k, 1 spin, seed 4\n")
        fh.write("# (synth.scaled_cell(2000, seed=4, kgrid=(4, 4, 4), nspin=1, ill_conditioned=False)),\n")
        fh.write("# written by tests/golden/make_mixed_n2000_oracle.py (oracle/ only: Sec. 3 Parts 1-4).\n")
        fh.write("# columns: problem (k index), m (kept overlap directions), band j, eps_j\n")
        for p, m, eps in res:
            for j, e in enumerate(eps):
                fh.write(f"{p} {m} {j} {e:.17e}\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
