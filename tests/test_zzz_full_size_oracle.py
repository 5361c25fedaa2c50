"""The headline workload at full size against the oracle's own full solve.

tests/golden/graded_c128_n4096_oracle_lambda.txt holds the eigenvalues of the
graded complex128 input of order 4096, computed by the oracle alone (the plain
method, Alg. 3.2 with the rotations of Alg. 3.1, round-robin order) and
written by tests/golden/make_graded_c128_n4096_oracle.py. The CPU test ties
the stored values to the input through invariants; the GPU test solves the
input in bench.py's configuration and compares. This file runs last, so a
failure under -x skips nothing else."""
import os

import numpy as np
import pytest

import synth
from tests._util import max_rel_err

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                    "graded_c128_n4096_oracle_lambda.txt")


def _gold():
    return np.loadtxt(GOLD, comments="#")


def test_stored_oracle_eigenvalues_fit_the_input():
    """The stored values belong to this input: one per column, the signs of J
    column by column, and sum lambda_i = trace(H) = sum_i J_ii ||g_i||^2 of the
    original G (the trace of H = G J G^* is invariant under the method's
    J-unitary transformations)."""
    lam = _gold()
    P = synth.make_workload("graded_c128_n4096_b64", precision="f64")
    assert lam.shape == (P.n,)
    assert np.all(np.sign(lam) == P.J)
    tr = float(np.sum(P.J * np.sum(np.abs(P.G) ** 2, axis=0)))
    scale = float(np.sum(np.abs(lam)))
    assert abs(np.sum(lam) - tr) <= 1e-12 * scale


def test_stored_values_come_from_the_oracle_alone():
    """The script that wrote the stored values imports only the oracle, the
    input generators and the standard library / numpy: no product code."""
    import ast

    src = os.path.join(os.path.dirname(GOLD), "make_graded_c128_n4096_oracle.py")
    mods = set()
    for node in ast.walk(ast.parse(open(src).read())):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            mods.add((node.module or "").split(".")[0])
    assert mods <= {"os", "sys", "time", "numpy", "oracle", "synth"}, mods


@pytest.mark.gpu
@pytest.mark.parametrize("gemm", [1, 2])  # all digits (the bench's form), hybrid
def test_headline_eigenvalues_match_the_full_oracle_solve(gemm):
    from tests.gpu_util import require_gpu, to_dev

    jj = require_gpu()
    import torch

    P = synth.make_workload("graded_c128_n4096_b64", precision="f64")
    ref = _gold()
    Gd = to_dev(P.G)
    with jj.Handle(P.m, P.n, jj.JJ_C128, block_width=16, gemm=gemm,
                   block_strategy=jj.JJ_BLOCK_ORIENTED) as h:
        info = h.jjacobi_solve(Gd, Gd.stride(1), P.J)
        lam = torch.empty(P.n, dtype=torch.float64, device="cuda")
        h.jjacobi_extract(lam)
    lam = lam.cpu().numpy()
    assert info.status == 0
    assert np.all(np.sign(lam) == P.J)
    # lambda sorted by value: which column carries which eigenvalue depends on
    # the order of the rotations (blocked here, column round robin in the oracle)
    assert max_rel_err(np.sort(lam), np.sort(ref)) <= 1e-10
