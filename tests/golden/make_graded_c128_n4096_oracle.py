"""Writes graded_c128_n4096_oracle_lambda.txt: the eigenvalues of the graded
complex128 workload of order 4096 (G = D1 B D2, B = Q |Lambda|^{1/2} W,
J = diag(+I_2560, -I_1536); the headline input) computed by the oracle alone.

The oracle here is the plain one-sided J-Jacobi method (Alg. 3.2 with the
rotations of Alg. 3.1) in round-robin order over single columns, run on all
host threads by oracle.solve_plain_threads, which returns the sequential
oracle's bits in that order. Only oracle/ computes; synth/ builds the seeded
input. Run from the repository root:

    python tests/golden/make_graded_c128_n4096_oracle.py

(about 40 minutes on 8 cores).
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                   "graded_c128_n4096_oracle_lambda.txt")


def main():
    P = synth.make_workload("graded_c128_n4096_b64", precision="f64")
    nt = len(os.sched_getaffinity(0))
    t0 = time.time()
    res = oracle.solve_plain_threads(P.G, P.J, nthreads=nt, max_sweeps=60)
    dt = time.time() - t0
    assert res["status"] == 0, res["status"]
    lam, _ = oracle.eigenpairs(res["Gt"], P.J)
    with open(OUT, "w") as f:
        f.write("# Eigenvalues lambda_i = J_ii ||g~_i||^2 of the graded complex128 workload of\n")
        f.write("# order 4096 (synth.make_workload('graded_c128_n4096_b64', precision='f64')),\n")
        f.write("# computed by the oracle: plain one-sided J-Jacobi (Alg. 3.2, rotations of\n")
        f.write("# Alg. 3.1), round-robin order over single columns, tol = 128 * 2^-53.\n")
        f.write(f"# Written by make_graded_c128_n4096_oracle.py: {res['sweeps']} sweeps, "
                f"{res['rotations']} rotations, {nt} threads, {dt:.0f} s.\n")
        f.write("# One value per line, in the input's column order.\n")
        for v in lam:
            f.write(repr(float(v)) + "\n")
    print(f"wrote {OUT}: {res['sweeps']} sweeps, {dt:.0f} s")


if __name__ == "__main__":
    main()
