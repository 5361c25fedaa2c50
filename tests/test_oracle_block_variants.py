"""Pins for the oracle's block-oriented (2B, Alg. 3.4 / Sec. 5.3) and
three-level (3F, 3B; Sec. 5.1-5.2, Algs. 3.3 and 5.1) references: they compute
the eigen-decomposition the plain method defines (Algs. 3.1/3.2), their pass
tables visit each pair exactly once, the inner partition respects the outer
block boundary, and a planted mistake (no whole-pivot pass) fails."""
from itertools import combinations

import numpy as np
import pytest

import oracle
import synth
from tests._util import eig_rel_tol, max_rel_err, orth_residual, reconstruction_residual


@pytest.mark.parametrize("ni,nj", [(4, 4), (5, 4), (1, 3), (7, 6)])
def test_block_oriented_pairs_visit_each_pair_once(ni, nj):
    whole = oracle.block_oriented_pairs(ni, nj, True)
    cross = oracle.block_oriented_pairs(ni, nj, False)
    k = ni + nj
    assert len(set(whole)) == len(whole) and set(map(tuple, map(sorted, whole))) == set(combinations(range(k), 2))
    assert set(cross) == {(r, ni + s) for r in range(ni) for s in range(nj)} and len(cross) == ni * nj
    tab = oracle.pass_table(k, cross)
    got = [tuple(p) for step in tab for p in step if p[0] < k and p[1] < k]
    assert got == cross


@pytest.mark.parametrize("ni,nj,ib", [(16, 16, 4), (13, 12, 4), (9, 8, 16), (3, 5, 2)])
def test_inner_partition_respects_block_boundary(ni, nj, ib):
    sizes = oracle._inner_blocks(ni, nj, ib)
    nb = len(sizes) // 2
    assert sum(sizes[:nb]) == ni and sum(sizes[nb:]) == nj
    for half in (sizes[:nb], sizes[nb:]):  # uniform partitions (3.3) of each block
        assert max(half) - min(half) <= 1
    assert all(s >= 1 for s in sizes)
    if nb < min(ni, nj):  # not limited by the smaller block: inner blocks of at most ib
        assert max(sizes) <= ib


@pytest.mark.parametrize("cplx,strategy", [(True, 0), (False, 1), (True, 1)])
def test_block_oriented_reference_matches_plain(cplx, strategy):
    P = (synth.make_workload("plain_c128_n128", n=48) if cplx
         else synth.make_workload("blocked_f64_n2048_b32", n=50))
    ref = oracle.solve_plain(P.G, P.J)
    got = oracle.solve_block_oriented(P.G, P.J, 5, strategy=strategy)
    tol = eig_rel_tol(P.G)
    assert got["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= tol
    assert orth_residual(got["U"]) <= 8 * oracle.TOL_DEFAULT
    assert reconstruction_residual(P.G, P.J, got["lam"], got["U"]) <= 1e-12


@pytest.mark.parametrize("variant", ["F", "B"])
@pytest.mark.parametrize("cplx", [True, False])
def test_three_level_reference_matches_plain(variant, cplx):
    P = (synth.make_workload("plain_c128_n128", n=46) if cplx
         else synth.make_workload("threelevel_f64_n16384_b128", n=52))
    ref = oracle.solve_plain(P.G, P.J)
    got = oracle.solve_three_level(P.G, P.J, 11, 3, variant=variant)
    tol = eig_rel_tol(P.G)
    assert got["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= tol
    if P.lam_exact is not None:
        assert max_rel_err(got["lam"], P.lam_exact) <= tol
    assert orth_residual(got["U"]) <= 8 * oracle.TOL_DEFAULT


def test_mutation_no_whole_pivot_pass_breaks_block_oriented():
    """Without the first step's whole-pivot pass, column pairs inside a block are
    never rotated: the sweeps stop with non-orthogonal columns."""
    P = synth.make_workload("plain_c128_n128", n=40)
    ref = oracle.solve_plain(P.G, P.J)
    bad = oracle.solve_block_oriented(P.G, P.J, 5, whole_first=False, max_sweeps=30)
    assert bad["status"] != 0 or max_rel_err(bad["lam"], ref["lam"]) > 1e-6


def _pivot_with_diagonal_blocks(rng, m, ni, nj, cplx):
    """[G_i G_j] whose blocks have orthogonal columns: A_P has the form (3.7)."""
    def block(w):
        Z = rng.standard_normal((m, w)) + (1j * rng.standard_normal((m, w)) if cplx else 0)
        Q, _ = np.linalg.qr(Z)
        return Q * (10.0 ** rng.uniform(-2, 2, size=w))[None, :]
    Gi, Gj = block(ni), block(nj)
    # mix the two blocks (the pair is not yet orthogonal across blocks)
    Gj = Gj + Gi @ (0.3 * rng.standard_normal((ni, nj)))
    Q, Rr = np.linalg.qr(Gj)
    Gj = Q * np.abs(np.diag(Rr))[None, :]  # re-orthogonalize within block j, keep the mixing
    return Gi, Gj


@pytest.mark.parametrize("cplx", [True, False])
def test_special_cholesky_is_the_cholesky_factor(cplx):
    rng = np.random.default_rng(21 + cplx)
    for ni, nj in ((5, 5), (6, 4), (3, 7)):
        Gi, Gj = _pivot_with_diagonal_blocks(rng, 30, ni, nj, cplx)
        A = np.concatenate([Gi, Gj], axis=1)
        A = A.conj().T @ A
        lam_i = np.sum(np.abs(Gi) ** 2, axis=0)
        lam_j = np.sum(np.abs(Gj) ** 2, axis=0)
        R = oracle.cholesky_special(lam_i, lam_j, Gi.conj().T @ Gj)
        scale = np.sqrt(np.outer(np.diag(A).real, np.diag(A).real))
        assert np.max(np.abs(R.conj().T @ R - A) / scale) <= 1e-12
        Rstd = oracle.cholesky_upper(A)  # unique with a positive diagonal
        assert np.max(np.abs(R - Rstd)) <= 1e-10 * np.max(np.abs(Rstd))
        try:  # the planted mistake: either the (3.11) block is no longer positive definite
            bad = oracle.cholesky_special(lam_i, lam_j, Gi.conj().T @ Gj, mutation=1)
        except np.linalg.LinAlgError:
            continue
        assert np.max(np.abs(bad.conj().T @ bad - A) / scale) > 1e-3  # or R^* R is not A


@pytest.mark.parametrize("cplx", [True, False])
def test_full_block_with_special_cholesky_matches_plain(cplx):
    P = (synth.make_workload("plain_c128_n128", n=40) if cplx
         else synth.make_workload("blocked_f64_n2048_b32", n=44))
    ref = oracle.solve_plain(P.G, P.J)
    got = oracle.solve_blocked_special(P.G, P.J, 5)
    assert got["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= eig_rel_tol(P.G)
    assert orth_residual(got["U"]) <= 8 * oracle.TOL_DEFAULT
