"""Pins for the CPU oracle: every oracle function checked against something other
than itself (closed forms, invariants, constructions with known eigenvalues,
LAPACK special cases, brute force), and planted mistakes shown to fail them."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests._util import (U64, eig_rel_tol, kappa_scaled, max_rel_err, orth_residual,
                         reconstruction_residual)


def _rand_pair(rng, m, cplx):
    if cplx:
        return rng.standard_normal((m, 2)) + 1j * rng.standard_normal((m, 2))
    return rng.standard_normal((m, 2))


def _pencil_eigs_2x2(A, j1, j2):
    """Roots of det(A - lambda J) = 0 for 2x2 A: the closed form of the 2x2 pair.

    j1 j2 lam^2 - (a11 j2 + a22 j1) lam + (a11 a22 - |a12|^2) = 0."""
    a11, a22 = A[0, 0].real, A[1, 1].real
    det = a11 * a22 - abs(A[0, 1]) ** 2
    qa, qb, qc = j1 * j2, -(a11 * j2 + a22 * j1), det
    disc = math.sqrt(qb * qb - 4 * qa * qc)
    q = -0.5 * (qb + math.copysign(disc, qb))  # stable quadratic roots
    return sorted([q / qa, qc / q])


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("jj", [(1, 1), (1, -1), (-1, 1), (-1, -1)])
def test_two_by_two_closed_form(cplx, jj):
    rng = np.random.default_rng(7 + jj[0] + 3 * jj[1] + 10 * cplx)
    for trial in range(20):
        G = _rand_pair(rng, 9, cplx)
        G[:, 1] *= 10.0 ** rng.uniform(-3, 3)
        A = G.conj().T @ G
        res = oracle.solve_plain(G, list(jj), max_sweeps=5)
        assert res["status"] == 0
        lam = sorted(float(x) for x in res["lam"])
        ref = _pencil_eigs_2x2(A, *jj)
        for a, b in zip(lam, ref):
            assert abs(a - b) <= 1e-13 * abs(b), (lam, ref)
        # one rotation annihilates a_rs (columns orthogonal after sweep 1)
        one = oracle.solve_plain(G, list(jj), max_sweeps=1)
        g = one["Gt"]
        off = abs(np.vdot(g[:, 0], g[:, 1])) / (np.linalg.norm(g[:, 0]) * np.linalg.norm(g[:, 1]))
        assert off < 64 * U64


def _rotation_matrix(par, hyp):
    """W_P of the modified rotation: g_r' = e c g_r - hyp s g_s, g_s' = e s g_r + c g_s."""
    c, s, e = float(par["c"]), float(par["s"]), par["e"]
    return np.array([[e * c, e * s], [-hyp * s, c]], dtype=np.complex128)


@pytest.mark.parametrize("hyp", [1, -1])
def test_rotation_is_j_unitary_and_diagonalizes(hyp):
    rng = np.random.default_rng(11 + hyp)
    Jp = np.diag([1.0, float(hyp)])
    for trial in range(200):
        G = _rand_pair(rng, 5, True)
        A = G.conj().T @ G
        par = oracle.rotation(A[0, 0].real, A[1, 1].real, A[0, 1], hyp)
        assert par is not None
        W = _rotation_matrix(par, hyp)
        assert np.abs(W.conj().T @ Jp @ W - Jp).max() <= 8 * U64 * np.abs(W).max() ** 2
        B = W.conj().T @ A @ W
        scale = math.sqrt(abs(B[0, 0].real * B[1, 1].real))
        assert abs(B[0, 1]) <= 64 * U64 * np.abs(W).max() ** 2 * np.abs(A).max() + 0 * scale
        # tracked diagonal (reading of the d_rr update): d' = diag(W^* A W)
        assert abs(float(par["d_r"]) - B[0, 0].real) <= 1e-13 * abs(B[0, 0].real) + 1e-13 * np.abs(A).max()
        assert abs(float(par["d_s"]) - B[1, 1].real) <= 1e-13 * abs(B[1, 1].real) + 1e-13 * np.abs(A).max()


def test_rotation_edge_cases():
    # Re a_rs = 0: sgn(0) = +1, e^{i alpha} = i
    par = oracle.rotation(2.0, 1.0, 0.5j, 1)
    assert par is not None and abs(par["e"] - 1j) < 1e-15
    # theta = 0 (a_rr = a_ss, trig): t = 1, a 45 degree rotation
    par = oracle.rotation(1.0, 1.0, 0.25, 1)
    assert abs(float(par["t"]) - 1.0) < 1e-15
    # huge theta: first-order branch, no overflow
    par = oracle.rotation(1e200, 1.0, 1e-120, 1)
    assert par is not None and np.isfinite(float(par["t"])) and abs(float(par["t"])) < 1e-300
    # not positive definite in the hyperbolic case: |a_rs| > (a_rr + a_ss)/2
    assert oracle.rotation(1.0, 1.0, 1.5, -1) is None


def test_known_by_construction_complex_n128():
    P = synth.make_workload("plain_c128_n128")
    tol = eig_rel_tol(P.G)
    for prec in ("f64", "ld"):
        res = oracle.solve_plain(P.G, P.J, precision=prec)
        assert res["status"] == 0
        assert max_rel_err(res["lam"], P.lam_exact) <= tol
        assert orth_residual(res["U"]) <= 4 * oracle.TOL_DEFAULT


def test_known_by_construction_real():
    P = synth.make_workload("blocked_f64_n2048_b32", n=96)
    tol = eig_rel_tol(P.G)
    res = oracle.solve_plain(P.G, P.J)
    assert res["status"] == 0
    assert max_rel_err(res["lam"], P.lam_exact) <= tol


def test_long_double_and_double_agree():
    P = synth.make_workload("plain_c128_n128", n=48)
    a = oracle.solve_plain(P.G, P.J, precision="f64")
    b = oracle.solve_plain(P.G, P.J, precision="ld")
    assert max_rel_err(a["lam"], b["lam"].astype(np.float64)) <= eig_rel_tol(P.G)


@pytest.mark.parametrize("sign", [1, -1])
@pytest.mark.parametrize("cplx", [True, False])
def test_definite_case_is_hestenes_svd(sign, cplx):
    """J = +-I reduces to the one-sided Hestenes SVD: lambda = +-sigma(G)^2 (LAPACK)."""
    rng = np.random.default_rng(3)
    m, n = 50, 40
    G = rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cplx else 0)
    res = oracle.solve_plain(G, [sign] * n)
    assert res["status"] == 0
    sig = np.linalg.svd(G, compute_uv=False)
    assert max_rel_err(res["lam"], sign * sig ** 2) <= 1e-13


@pytest.mark.parametrize("n", [3, 5, 6])
def test_brute_force_mpmath(n):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    P = synth.make_problem(n, True, (n + 1) // 2, (1e-2, 1e2), 2 * n, 1.5, seed=(77, n))
    H = mp.matrix(n, n)
    G, J = P.G, P.J
    for a in range(n):
        for b in range(n):
            H[a, b] = mp.fsum(mp.mpc(G[a, k]) * int(J[k]) * mp.conj(mp.mpc(G[b, k]))
                              for k in range(n))
    ev = mp.eighe(H, eigvals_only=True) if hasattr(mp, "eighe") else mp.eig(H)[0]
    ref = sorted(float(mp.re(x)) for x in ev)
    for prec, tol in (("ld", 4 * 2.0 ** -63 * kappa_scaled(G) + 1e-17), ("f64", eig_rel_tol(G))):
        res = oracle.solve_plain(G, J, precision=prec)
        assert max_rel_err(res["lam"].astype(np.float64), ref) <= max(tol, 1e-15)


def test_accumulated_w_is_j_unitary_and_reproduces_gt():
    P = synth.make_workload("plain_c128_n128", n=40)
    res = oracle.solve_plain(P.G, P.J, accumulate=True)
    W = res["W"]
    Jd = np.diag(P.J.astype(np.float64))
    wmax = np.abs(W).max()
    assert np.abs(W.conj().T @ Jd @ W - Jd).max() <= 1e3 * U64 * wmax ** 2
    assert np.abs(P.G @ W - res["Gt"]).max() <= 1e3 * U64 * wmax * np.abs(P.G).max()
    assert reconstruction_residual(P.G, P.J, res["lam"], res["U"]) <= 1e-12


def test_orders_agree():
    P = synth.make_workload("plain_c128_n128", n=64)
    tol = eig_rel_tol(P.G)
    base = oracle.solve_plain(P.G, P.J, order=oracle.ORDER_ROW_CYCLIC)
    for order in (oracle.ORDER_COLUMN_CYCLIC, oracle.ORDER_ROUND_ROBIN):
        other = oracle.solve_plain(P.G, P.J, order=order)
        assert other["status"] == 0
        assert max_rel_err(other["lam"], base["lam"]) <= tol


def test_odd_order_round_robin():
    P = synth.make_workload("plain_c128_n128", n=33)
    a = oracle.solve_plain(P.G, P.J, order=oracle.ORDER_ROUND_ROBIN)
    assert a["status"] == 0
    assert max_rel_err(a["lam"], P.lam_exact) <= eig_rel_tol(P.G)


def test_invalid_arguments():
    G = np.eye(4)
    assert oracle.solve_plain(G, [1, 1, 2, 1])["status"] == 1
    assert oracle.solve_plain(np.ones((2, 3)), [1, 1, 1])["status"] == 1


def test_rank_deficient_loses_definiteness_or_stalls():
    """A singular G (not of full column rank) violates the method's premise (2.6)."""
    rng = np.random.default_rng(5)
    G = rng.standard_normal((8, 4))
    G[:, 3] = G[:, 0] + G[:, 1]
    res = oracle.solve_plain(G, [1, -1, 1, -1], max_sweeps=30)
    assert res["status"] in (2, 3) or np.min(np.abs(res["lam"])) < 1e-10


# ---------------------------------------------------------------------------
# Planted mistakes: each plausible error in the printed formulas fails a pin
# ---------------------------------------------------------------------------

def test_mutation_literal_hyp_sign_breaks_j_unitarity():
    rng = np.random.default_rng(1)
    G = _rand_pair(rng, 6, True)
    A = G.conj().T @ G
    par = oracle.rotation(A[0, 0].real, A[1, 1].real, A[0, 1], -1, mutation=1)
    Jp = np.diag([1.0, -1.0])
    if par is None:
        return  # the literal sign also fails by breaking positivity
    W = _rotation_matrix(par, -1)
    assert np.abs(W.conj().T @ Jp @ W - Jp).max() > 1e-3


def test_mutation_literal_d_update_breaks_tracking():
    rng = np.random.default_rng(2)
    G = _rand_pair(rng, 6, True)
    A = G.conj().T @ G
    par = oracle.rotation(A[0, 0].real, A[1, 1].real, A[0, 1], 1, mutation=2)
    W = _rotation_matrix(par, 1)
    B = W.conj().T @ A @ W
    assert abs(float(par["d_r"]) - B[0, 0].real) > 1e-6 * abs(B[0, 0].real)


def test_mutation_duplicated_column_write_breaks_eigenvalues():
    P = synth.make_workload("plain_c128_n128", n=16)
    res = oracle.solve_plain(P.G, P.J, mutation=3, max_sweeps=10)
    bad = res["status"] != 0 or max_rel_err(res["lam"], P.lam_exact) > 1e-6
    assert bad


@pytest.mark.parametrize("order", [oracle.ORDER_ROW_CYCLIC, oracle.ORDER_ROUND_ROBIN])
def test_state_between_sweeps_is_g_alone(order):
    """Alg. 3.2 recomputes the diagonal at the start of every sweep, so the
    state between sweeps is the current G~ alone: a solve capped after k sweeps
    and resumed from its G~ gives the bits of the uninterrupted solve. (This is
    what makes a capped solve a checkpoint.)"""
    P = synth.make_workload("plain_c128_n128", n=40)
    full = oracle.solve_plain(P.G, P.J, order=order)
    part = oracle.solve_plain(P.G, P.J, order=order, max_sweeps=3)
    assert part["status"] == 2 and full["sweeps"] > 3
    rest = oracle.solve_plain(part["Gt"], P.J, order=order)
    assert rest["status"] == 0 and part["sweeps"] + rest["sweeps"] == full["sweeps"]
    assert np.array_equal(rest["Gt"], full["Gt"])


@pytest.mark.parametrize("hyp", [1, -1])
def test_rotation_across_column_scales(hyp):
    """Columns of very different lengths (the graded inputs' situation, here
    up to 1e120 apart): the rotation stays finite and J-unitary, and the
    rotated pair is orthogonal relative to its own column lengths. The method
    works with squared norms, so the range is the one where products of two
    squared column norms stay in FP64 (norms within about 1e+-75)."""
    rng = np.random.default_rng(21 + hyp)
    Jp = np.diag([1.0, float(hyp)])
    for e1 in (-60, -30, -5, 0, 5, 30, 60):
        for e2 in (-60, -8, 0, 8, 60):
            G = _rand_pair(rng, 6, True)
            G[:, 0] *= 10.0 ** e1
            G[:, 1] *= 10.0 ** e2
            A = G.conj().T @ G
            par = oracle.rotation(A[0, 0].real, A[1, 1].real, A[0, 1], hyp)
            assert par is not None
            W = _rotation_matrix(par, hyp)
            assert np.all(np.isfinite(W))
            assert np.abs(W.conj().T @ Jp @ W - Jp).max() <= 8 * U64 * np.abs(W).max() ** 2
            Gt = G @ W
            n0, n1 = np.linalg.norm(Gt[:, 0]), np.linalg.norm(Gt[:, 1])
            assert abs(np.vdot(Gt[:, 0], Gt[:, 1])) <= 64 * U64 * np.abs(W).max() ** 2 * max(
                n0 * n1, abs(A[0, 1]))
