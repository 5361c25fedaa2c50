"""GPU parity of the plain (non-blocked) path against the CPU oracle, through
the C ABI: eigenvalues, one sweep element by element, eigenvectors, edge cases."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import eig_rel_tol, max_rel_err, orth_residual, reconstruction_residual
from tests.gpu_util import col_rel_err, require_gpu, solve_gpu, to_dev

pytestmark = pytest.mark.gpu


def test_plain_c128_n128_matches_oracle():
    """The full plain complex128 n = 128 workload."""
    require_gpu()
    P = synth.make_workload("plain_c128_n128")
    ref = oracle.solve_plain(P.G, P.J)
    got = solve_gpu(P.G, P.J, want_U=True)
    tol = eig_rel_tol(P.G)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= tol
    assert max_rel_err(got["lam"], P.lam_exact) <= tol
    assert np.array_equal(np.sign(got["lam"]), P.J)
    assert orth_residual(got["U"]) <= 8 * oracle.TOL_DEFAULT
    assert reconstruction_residual(P.G, P.J, got["lam"], got["U"]) <= 1e-12


@pytest.mark.parametrize("cplx", [True, False])
def test_plain_one_sweep_elementwise(cplx):
    """After exactly one round-robin sweep the GPU factor equals the oracle's
    (same ordering: Alg. 4.3 over columns), column by column."""
    require_gpu()
    name = "plain_c128_n128" if cplx else "blocked_f64_n2048_b32"
    P = synth.make_workload(name, n=64)
    ref = oracle.solve_plain(P.G, P.J, max_sweeps=1, order=oracle.ORDER_ROUND_ROBIN)
    got = solve_gpu(P.G, P.J, max_sweeps=1, allow=(0, 2))
    assert got["info"]["sweeps"] == 1
    assert col_rel_err(got["Gt"], ref["Gt"]) <= 1e-11
    assert got["info"]["rotations"] == ref["rotations"]


@pytest.mark.parametrize("m,n", [(33, 33), (80, 48), (5, 2), (2, 2), (3, 1), (257, 255)])
def test_plain_ragged_and_tall(m, n):
    require_gpu()
    P = synth.make_problem(n, True, max(1, n // 3), (1e-2, 1e2), 2 * n, 1.5, seed=(5, m, n), m=m)
    ref = oracle.solve_plain(P.G, P.J)
    got = solve_gpu(P.G, P.J)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= eig_rel_tol(P.G)


def test_plain_real_matches_construction():
    require_gpu()
    P = synth.make_workload("blocked_f64_n2048_b32", n=128)
    got = solve_gpu(P.G, P.J)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], P.lam_exact) <= eig_rel_tol(P.G)


def test_plain_unsorted_j_keeps_column_order():
    require_gpu()
    P = synth.make_workload("plain_c128_n128", n=40)
    perm = np.random.default_rng(1).permutation(40)
    G = np.asfortranarray(P.G[:, perm])
    J = P.J[perm]
    got = solve_gpu(G, J)
    ref = oracle.solve_plain(G, J)
    # J-unitary transformations keep each column's sign (Sec. 2.3); which
    # eigenvalue of that sign ends in which column depends on the rotation
    # order, so the values are compared as sorted sets.
    assert np.array_equal(np.sign(got["lam"]), J)
    assert max_rel_err(got["lam"], ref["lam"]) <= eig_rel_tol(G)


def test_extract_sorted_with_vectors():
    require_gpu()
    P = synth.make_workload("plain_c128_n128", n=32)
    got = solve_gpu(P.G, P.J, want_U=True, sort=1)
    lam = got["lam"]
    assert np.all(np.diff(lam) >= 0)
    U = got["U"]
    assert np.allclose(np.linalg.norm(U, axis=0), 1.0, atol=1e-14)
    # U's columns are the normalized columns of G~, in the order of lambda
    Gt = got["Gt"]
    nrm = np.linalg.norm(Gt, axis=0)
    order = np.argsort(P.J * nrm ** 2, kind="stable")
    assert np.allclose(U, Gt[:, order] / nrm[order], atol=1e-14)


def test_solve_host_end_to_end():
    jj = require_gpu()
    P = synth.make_workload("plain_c128_n128", n=48)
    ref = oracle.solve_plain(P.G, P.J)
    with jj.Handle(P.m, P.n, jj.JJ_C128) as h:
        lam, U, info = h.jjacobi_solve_host(P.G, P.J, want_U=True)
    assert info.status == 0
    assert max_rel_err(lam, ref["lam"]) <= eig_rel_tol(P.G)
    assert orth_residual(U) <= 8 * oracle.TOL_DEFAULT


def test_error_paths():
    jj = require_gpu()
    P = synth.make_workload("plain_c128_n128", n=16)
    G = P.G.copy()
    G[3, 4] = np.nan
    got = solve_gpu(G, P.J, allow=(jj.JJ_NONFINITE,))
    assert got["info"]["status"] == jj.JJ_NONFINITE
    got = solve_gpu(P.G, P.J, max_sweeps=2, allow=(jj.JJ_NOT_CONVERGED,))
    assert got["info"]["status"] == jj.JJ_NOT_CONVERGED and got["info"]["sweeps"] == 2
    bad = P.J.copy()
    bad[0] = 3
    with pytest.raises(jj.JJError) as e:
        solve_gpu(P.G, bad)
    assert e.value.status == jj.JJ_INVALID_ARG
    # extract before any solve
    import torch
    with jj.Handle(P.m, P.n, jj.JJ_C128) as h:
        lam = torch.empty(P.n, dtype=torch.float64, device="cuda")
        with pytest.raises(jj.JJError) as e:
            h.jjacobi_extract(lam)
        assert e.value.status == jj.JJ_NOT_SOLVED


def test_rank_deficient_reports_status():
    jj = require_gpu()
    rng = np.random.default_rng(5)
    G = rng.standard_normal((12, 6))
    G[:, 5] = G[:, 0] - 2 * G[:, 1]
    got = solve_gpu(np.asfortranarray(G), [1, -1, 1, -1, 1, -1], max_sweeps=30,
                    allow=(0, jj.JJ_NOT_POSDEF, jj.JJ_NOT_CONVERGED, jj.JJ_NONFINITE))
    st = got["info"]["status"]
    assert st in (jj.JJ_NOT_POSDEF, jj.JJ_NOT_CONVERGED, jj.JJ_NONFINITE) or \
        np.min(np.abs(got["lam"])) < 1e-10
