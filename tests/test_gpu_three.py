"""Three-level form (Sec. 5.1, case 3F: the inner J-Jacobi of every outer pivot
is itself the blocked method, Alg. 3.3 on R) against the oracle, against
eigenvalues known by construction and against the two-level form."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import eig_rel_tol, max_rel_err, orth_residual, reconstruction_residual
from tests.gpu_util import require_gpu, solve_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("gemm", [0, 1, 2])
@pytest.mark.parametrize("order", [0, 1])
def test_three_level_real_matches_oracle(gemm, order):
    require_gpu()
    P = synth.make_workload("threelevel_f64_n16384_b128", n=256)
    ref = oracle.solve_plain(P.G, P.J)
    # outer pivots of 64 columns, inner blocks of 8: 8 inner blocks per pivot
    got = solve_gpu(P.G, P.J, block_width=32, inner_block_width=8, gemm=gemm, order=order,
                    want_U=True)
    tol = eig_rel_tol(P.G)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= tol
    assert max_rel_err(got["lam"], P.lam_exact) <= tol
    assert orth_residual(got["U"]) <= 8 * oracle.TOL_DEFAULT
    assert reconstruction_residual(P.G, P.J, got["lam"], got["U"]) <= 1e-12


@pytest.mark.parametrize("gemm", [0, 1])
def test_three_level_complex_ragged(gemm):
    """Complex, ragged outer and inner partitions (150 columns, b = 20: pivots
    of 36-40 columns; inner blocks of 6)."""
    require_gpu()
    P = synth.make_workload("plain_c128_n128", n=150)
    ref = oracle.solve_plain(P.G, P.J)
    got = solve_gpu(P.G, P.J, block_width=20, inner_block_width=6, gemm=gemm)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= eig_rel_tol(P.G)
    assert max_rel_err(got["lam"], P.lam_exact) <= eig_rel_tol(P.G)


def test_three_level_agrees_with_two_level_wide_pivot():
    """Outer pivots of 256 columns (the 16 384-column workload's b = 128) with
    inner blocks of 16, at n = 1024: the outer contractions run as digit
    products over 4 x 4 tiles of 64 positions, the inner ones as single-tile
    digit products; eigenvalues by construction and against the two-level
    form in FP64."""
    require_gpu()
    P = synth.make_workload("threelevel_f64_n16384_b128", n=1024)
    three = solve_gpu(P.G, P.J, block_width=128, inner_block_width=16, gemm=1)
    two = solve_gpu(P.G, P.J, block_width=128, gemm=0)
    tol = eig_rel_tol(P.G)
    assert three["info"]["status"] == 0 and two["info"]["status"] == 0
    assert max_rel_err(three["lam"], P.lam_exact) <= tol
    assert max_rel_err(three["lam"], two["lam"]) <= tol


@pytest.mark.parametrize("gemm", [0, 1, 2])
def test_three_level_block_oriented_matches_oracle(gemm):
    """3B (Sec. 5.2-5.3, Alg. 5.1): in the first step of a sweep one
    block-oriented inner pass over every inner block pair of the pivot, in the
    other steps one pass over the cross pairs (inner blocks of block i against
    inner blocks of block j) only."""
    jj = require_gpu()
    P = synth.make_workload("threelevel_f64_n16384_b128", n=256)
    ref = oracle.solve_plain(P.G, P.J)
    got = solve_gpu(P.G, P.J, block_width=32, inner_block_width=8, gemm=gemm,
                    block_strategy=jj.JJ_BLOCK_ORIENTED, want_U=True)
    tol = eig_rel_tol(P.G)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= tol
    assert max_rel_err(got["lam"], P.lam_exact) <= tol
    assert orth_residual(got["U"]) <= 8 * oracle.TOL_DEFAULT
    assert reconstruction_residual(P.G, P.J, got["lam"], got["U"]) <= 1e-12


def test_three_level_block_oriented_complex_ragged_wide():
    """3B with unequal outer blocks and ragged inner blocks (complex, 150
    columns, b = 20, inner 6), and with 256-column outer pivots (n = 1024)."""
    jj = require_gpu()
    P = synth.make_workload("plain_c128_n128", n=150)
    ref = oracle.solve_plain(P.G, P.J)
    got = solve_gpu(P.G, P.J, block_width=20, inner_block_width=6, gemm=1,
                    block_strategy=jj.JJ_BLOCK_ORIENTED)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= eig_rel_tol(P.G)
    Q = synth.make_workload("threelevel_f64_n16384_b128", n=1024)
    w = solve_gpu(Q.G, Q.J, block_width=128, inner_block_width=16, gemm=1,
                  block_strategy=jj.JJ_BLOCK_ORIENTED)
    assert w["info"]["status"] == 0
    assert max_rel_err(w["lam"], Q.lam_exact) <= eig_rel_tol(Q.G)


def test_three_level_inner_width_not_below_pivot_is_two_level():
    """inner_block_width >= half the pivot: the two-level form runs (same bits)."""
    require_gpu()
    P = synth.make_workload("blocked_f64_n2048_b32", n=96)
    a = solve_gpu(P.G, P.J, block_width=8, inner_block_width=8, gemm=0)
    b = solve_gpu(P.G, P.J, block_width=8, gemm=0)
    assert np.array_equal(a["Gt"], b["Gt"])
