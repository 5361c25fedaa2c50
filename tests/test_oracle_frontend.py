"""Pins of the front-end oracle (H -> G, J of Sec. 2.2 and the zero-eigenvalue
completion after (2.11)) against textbook special cases, closed forms,
Sylvester's law of inertia, LAPACK eigenvalues and a planted mistake."""
import numpy as np
import pytest

import oracle
from oracle import frontend

EPS = 2.0 ** -53


def _herm(n, cplx, rng):
    X = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    return (X + X.conj().T) / 2


def _known(n, cplx, rng, lam):
    """H = Q diag(lam) Q^* with Q Haar-distributed, made exactly Hermitian."""
    X = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    Q, R = np.linalg.qr(X)
    Q = Q * (np.diag(R) / np.abs(np.diag(R)))
    H = (Q * lam) @ Q.conj().T
    return (H + H.conj().T) / 2


def _recon(f, H):
    G, J = f["G"], f["J"]
    return np.max(np.abs(G @ (J[:, None] * G.conj().T) - H)) / np.max(np.abs(H))


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("sign", [1, -1])
def test_definite_h_is_pivoted_cholesky(cplx, sign):
    """A definite H takes only 1x1 pivots (its largest entry lies on the
    diagonal), each the largest diagonal entry of the Schur complement; G in
    the pivot order is then the Cholesky factor of sign * P H P^T."""
    rng = np.random.default_rng(11 + cplx)
    n = 24
    X = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    H = sign * (X @ X.conj().T + n * np.eye(n))
    H = (H + H.conj().T) / 2
    f = frontend.factor_gj(H)
    assert f["rank"] == n and f["block_sizes"] == [1] * n
    assert np.all(f["J"] == sign)
    Hp = H[f["perm"]][:, f["perm"]]
    L = np.linalg.cholesky(sign * Hp)
    assert np.max(np.abs(f["Gp"] - L)) <= 1e-13 * np.max(np.abs(L))
    # the pivot order is diagonal pivoting: each pivot is the largest diagonal
    # entry of its Schur complement
    A = sign * Hp.copy()
    for k in range(n):
        assert np.real(A[k, k]) >= np.max(np.real(np.diag(A)[k:])) * (1 - 1e-12)
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:]) / A[k, k]


@pytest.mark.parametrize("H, lam", [
    (np.array([[0.0, 1.0], [1.0, 0.0]]), [-1.0, 1.0]),
    (np.array([[0.0, 1j], [-1j, 0.0]]), [-1.0, 1.0]),
    (np.array([[1.0, 2.0], [2.0, 1.0]]), [-1.0, 3.0]),
])
def test_two_by_two_pivots_closed_form(H, lam):
    """Indefinite 2x2 matrices whose diagonal is below alpha times the
    off-diagonal take one 2x2 pivot; G J G^* = H and the J-Jacobi eigenvalues
    are the closed-form ones."""
    f = frontend.factor_gj(H)
    assert f["block_sizes"] == [2]
    assert sorted(f["J"].tolist()) == [-1, 1]
    assert _recon(f, H) <= 8 * EPS
    res = frontend.eigh_via_jjacobi(H)
    assert np.allclose(np.sort(res["lam"]), lam, rtol=4 * EPS, atol=0)


def test_alpha_threshold_decides_the_pivot_size():
    """H = [[a, 1], [1, 0]]: a 1x1 pivot when a >= alpha = (1 + sqrt 17)/8
    (about 0.6404), a 2x2 pivot when a is just below it."""
    assert abs(frontend.ALPHA_BUNCH_PARLETT - 0.6403882032022076) < 1e-15
    for a, sizes in ((0.65, [1, 1]), (0.63, [2])):
        H = np.array([[a, 1.0], [1.0, 0.0]])
        f = frontend.factor_gj(H)
        assert f["block_sizes"] == sizes
        assert _recon(f, H) <= 8 * EPS
        assert sorted(f["J"].tolist()) == [-1, 1]  # det H = -1 < 0


@pytest.mark.parametrize("cplx", [False, True])
def test_random_indefinite_reconstruction_inertia_structure(cplx):
    """Random indefinite H: G J G^* = H to a small multiple of n eps; J counts
    the positive and negative eigenvalues of H (Sylvester's law of inertia);
    G in the pivot order is lower block triangular with the blocks of D; every
    2x2 block of D is indefinite."""
    rng = np.random.default_rng(21 + cplx)
    n = 40
    H = _herm(n, cplx, rng)
    f = frontend.factor_gj(H)
    assert f["rank"] == n
    assert _recon(f, H) <= 64 * n * EPS
    ev = np.linalg.eigvalsh(H)
    assert np.sum(f["J"] > 0) == np.sum(ev > 0) and np.sum(f["J"] < 0) == np.sum(ev < 0)
    assert 2 in f["block_sizes"]  # random indefinite matrices need some 2x2 pivots
    Gp = f["Gp"]
    k = 0
    for s in f["block_sizes"]:
        assert np.all(Gp[:k, k:k + s] == 0)  # above the diagonal block
        k += s
    b = frontend.bunch_parlett(H)
    for E in b["blocks"]:
        if E.shape[0] == 2:
            assert np.real(np.linalg.det(E)) < 0


@pytest.mark.parametrize("cplx", [False, True])
def test_whole_method_recovers_known_eigenvalues(cplx):
    """H = Q diag(lam) Q^* with lam known, both signs, |lam| in [1, 100]: the
    front end and the plain J-Jacobi oracle give lam to ~ n eps ||H|| / |lam|_min,
    and eigenvectors with H u = lam u."""
    rng = np.random.default_rng(31 + cplx)
    n = 32
    lam = np.exp(rng.uniform(0, np.log(100), n)) * rng.choice([-1.0, 1.0], n)
    H = _known(n, cplx, rng, lam)
    res = frontend.eigh_via_jjacobi(H)
    assert res["status"] == 0 and res["rank"] == n
    assert np.max(np.abs(np.sort(res["lam"]) - np.sort(lam)) / np.abs(np.sort(lam))) <= 1e-11
    U = res["U"]
    assert np.max(np.abs(H @ U - U * res["lam"])) <= 1e-11 * np.max(np.abs(lam))
    assert np.max(np.abs(U.conj().T @ U - np.eye(n))) <= 1e-12


@pytest.mark.parametrize("cplx", [False, True])
def test_singular_h_rank_factor_and_zero_eigenvectors(cplx):
    """rank(H) = r < n: G is n x r of full column rank, the J-Jacobi eigenvalues
    are the r nonzero ones, and the completion gives n - r orthonormal vectors
    orthogonal to the others with H z = 0."""
    rng = np.random.default_rng(41 + cplx)
    n, r = 30, 22
    lam = np.zeros(n)
    lam[:r] = np.exp(rng.uniform(0, np.log(10), r)) * rng.choice([-1.0, 1.0], r)
    H = _known(n, cplx, rng, lam)
    f = frontend.factor_gj(H, rank_tol=1e-10)
    assert f["rank"] == r and f["G"].shape == (n, r)
    assert np.linalg.matrix_rank(f["G"]) == r
    res = frontend.eigh_via_jjacobi(H, rank_tol=1e-10)
    nz = np.sort(res["lam"][:r])
    assert np.max(np.abs(nz - np.sort(lam[:r])) / np.abs(np.sort(lam[:r]))) <= 1e-10
    assert np.all(res["lam"][r:] == 0)
    U = res["U"]
    Z = U[:, r:]
    assert np.max(np.abs(U.conj().T @ U - np.eye(n))) <= 1e-12
    assert np.max(np.abs(H @ Z)) <= 1e-12 * np.max(np.abs(H))


def test_zero_eigenvectors_complete_an_orthonormal_basis():
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((9, 4)) + 1j * rng.standard_normal((9, 4)))
    Z = frontend.zero_eigenvectors(U)
    assert Z.shape == (9, 5)
    B = np.concatenate([U, Z], axis=1)
    assert np.max(np.abs(B.conj().T @ B - np.eye(9))) <= 1e-14


def test_definite_pair_with_plain_solver_is_hestenes():
    """J = I after the front end (positive definite H): the one-sided method
    is Hestenes' SVD of the Cholesky factor, so lambda = sigma(G)^2 = eig(H)."""
    rng = np.random.default_rng(7)
    X = rng.standard_normal((16, 16))
    H = X @ X.T + np.eye(16)
    res = frontend.eigh_via_jjacobi(H)
    ev = np.linalg.eigvalsh(H)
    assert np.max(np.abs(np.sort(res["lam"]) - ev) / ev) <= 1e-13


def test_mutation_transposed_schur_update_breaks_complex_reconstruction():
    """A plausible mistake (C E^-1 C^T in place of C E^-1 C^* in the Schur
    complement) leaves real H untouched but fails complex H."""
    rng = np.random.default_rng(8)
    Hr = _herm(20, False, rng)
    Hc = _herm(20, True, rng)
    assert _recon(frontend.factor_gj(Hr, mutation=1), Hr) <= 64 * 20 * EPS
    assert _recon(frontend.factor_gj(Hc), Hc) <= 64 * 20 * EPS
    assert _recon(frontend.factor_gj(Hc, mutation=1), Hc) > 1e-3


def test_rejects_non_hermitian_and_handles_zero():
    with pytest.raises(ValueError):
        frontend.factor_gj(np.array([[1.0, 2.0], [0.0, 1.0]]))
    f = frontend.factor_gj(np.zeros((3, 3)))
    assert f["rank"] == 0 and f["G"].shape == (3, 0)
    res = frontend.eigh_via_jjacobi(np.zeros((3, 3)))
    assert np.all(res["lam"] == 0) and res["U"].shape == (3, 3)
