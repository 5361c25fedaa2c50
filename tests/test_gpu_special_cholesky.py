"""The full-block form with the special pivot factor of Sec. 3.3 on the GPU:
each sweep opens with a pass that diagonalizes every block's own Gram, and every
pivot's factor is R_ii = sqrt(Lambda_ii) (3.9), R_ij = R_ii^{-1} A_ij (3.10),
R_jj the Cholesky factor of Lambda_jj - R_ij^* R_ij (3.11). Parity with the
oracle's reference of the same algorithm and with the plain method."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import eig_rel_tol, max_rel_err, orth_residual, reconstruction_residual
from tests.gpu_util import require_gpu, solve_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("recipe,n,b", [("plain_c128_n128", 128, 16), ("plain_c128_n128", 150, 11),
                                        ("blocked_f64_n2048_b32", 256, 32)])
@pytest.mark.parametrize("gemm", [0, 1])
def test_special_factor_matches_oracle(recipe, n, b, gemm):
    jj = require_gpu()
    P = synth.make_workload(recipe, n=n)
    ref = oracle.solve_blocked_special(P.G, P.J, b)
    plain = oracle.solve_plain(P.G, P.J)
    assert ref["status"] == 0
    got = solve_gpu(P.G, P.J, block_width=b, gemm=gemm, want_U=True,
                    pivot_factor=jj.JJ_PIVOT_SPECIAL)
    tol = eig_rel_tol(P.G)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= tol
    assert max_rel_err(got["lam"], plain["lam"]) <= tol
    assert orth_residual(got["U"]) <= 8 * oracle.TOL_DEFAULT
    assert reconstruction_residual(P.G, P.J, got["lam"], got["U"]) <= 1e-12


def test_special_factor_graded_held_to_published_bound():
    jj = require_gpu()
    P = synth.make_workload("graded_c128_n4096_b64", n=192)
    ref = oracle.solve_plain(P.G, P.J)
    for gemm in (1, 2):
        got = solve_gpu(P.G, P.J, block_width=16, gemm=gemm, pivot_factor=jj.JJ_PIVOT_SPECIAL)
        assert got["info"]["status"] == 0
        assert max_rel_err(got["lam"], ref["lam"]) <= 1e-10, gemm


def test_special_factor_refused_where_it_does_not_apply():
    jj = require_gpu()
    import torch

    for kw in (dict(block_strategy=jj.JJ_BLOCK_ORIENTED), dict(inner_block_width=8)):
        with pytest.raises(jj.JJError):
            with jj.Handle(96, 96, jj.JJ_C128, block_width=16, pivot_factor=jj.JJ_PIVOT_SPECIAL,
                           **kw) as h:
                G = torch.zeros((96, 96), dtype=torch.complex128, device="cuda").t()
                h.jjacobi_solve(G, 96, [1] * 96)
