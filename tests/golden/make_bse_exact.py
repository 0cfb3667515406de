"""Writes bse_exact_nk6250.txt: the 201 lowest eigenvalues of the synthetic
Eq. (1) Hamiltonian (seed 0, Nk = 6250, Nv = Nc = 4: N = 100000), exact in
FP64, from the structured oracle (Sylvester inertia counts of the block +
low-rank form and bisection; oracle/structured.py).  No dense matrix and no
part of the GPU path is involved.  Run from the repository root:

    python tests/golden/make_bse_exact.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle.structured as structured  # noqa: E402

SEED, NK, NV, NC, K = 0, 6250, 4, 4, 201


def main():
    lam = structured.lowest_eigenvalues(structured.bse_blocks(SEED, NK, NV, NC), K)
    with open(os.path.join(HERE, "bse_exact_nk6250.txt"), "w") as f:
        f.write("# The %d lowest eigenvalues of the synthetic Eq. (1) Hamiltonian, seed %d,\n"
                "# Nk = %d, Nv = %d, Nc = %d (N = %d), from the structured oracle\n"
                "# (Sylvester counts + bisection); written by make_bse_exact.py.\n"
                % (K, SEED, NK, NV, NC, NK * NV * NC))
        for x in lam:
            f.write("%.17e\n" % x)


if __name__ == "__main__":
    main()
