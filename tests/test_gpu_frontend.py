"""GPU front end H -> (G, J) (Sec. 2.2, (2.5)) against the oracle's
Bunch-Parlett factorization: the pivot sequence (permutation and block sizes)
and the signs J bit-exact, G per column to rounding (a 2x2 block's columns up
to the unit phase of its eigenvectors), H = G J G^* reconstructed, Sylvester's
inertia, the rank of a singular H, and the eigenvalues of H through the whole
method (front end, then the one-sided solve on the GPU)."""
import numpy as np
import pytest

from oracle import frontend
from tests._util import max_rel_err
from tests.gpu_util import require_gpu, solve_gpu

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


def _herm(n, cplx, rng):
    X = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    return (X + X.conj().T) / 2


def _known(n, cplx, rng, lam):
    X = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    Q, R = np.linalg.qr(X)
    Q = Q * (np.diag(R) / np.abs(np.diag(R)))
    H = (Q * lam) @ Q.conj().T
    return (H + H.conj().T) / 2


def _factor_gpu(H, rank_tol=0.0):
    jj = require_gpu()
    import torch

    Hd = torch.from_numpy(np.ascontiguousarray(H)).to("cuda")
    G, J, perm, psize, r = jj.jjacobi_factor(Hd, rank_tol)
    torch.cuda.synchronize()
    Gh = G.cpu().numpy() if r else np.zeros((H.shape[0], 0), dtype=H.dtype)
    return dict(G=Gh, J=J.astype(np.int64), perm=perm, psize=psize, rank=r)


def _block_sizes(psize):
    return [int(s) for s in psize if s != 0]


def _align_phases(Gg, Go, sizes):
    """The GPU's G with each column of a 2x2 block multiplied by the unit
    phase that best matches the oracle's (eigenvectors are unique up to it)."""
    Ga = Gg.copy()
    c = 0
    for s in sizes:
        if s == 2:
            for q in (c, c + 1):
                ph = np.vdot(Gg[:, q], Go[:, q])
                if ph != 0:
                    Ga[:, q] *= ph / abs(ph)
        c += s
    return Ga


def _check_against_oracle(H, rank_tol=None):
    g = _factor_gpu(H, 0.0 if rank_tol is None else rank_tol)
    o = frontend.factor_gj(H, rank_tol=rank_tol)
    n = H.shape[0]
    assert g["rank"] == o["rank"]
    assert np.array_equal(g["perm"], o["perm"])
    assert _block_sizes(g["psize"]) == o["block_sizes"]
    assert np.array_equal(g["J"], o["J"].astype(np.int64))
    r = o["rank"]
    if r:
        Ga = _align_phases(g["G"], o["G"], o["block_sizes"])
        scale = np.max(np.abs(o["G"]))
        assert np.max(np.abs(Ga - o["G"])) <= 64 * n * EPS * scale
        R = g["G"] @ (g["J"][:, None] * g["G"].conj().T)
        assert np.max(np.abs(R - H)) <= 64 * n * EPS * max(np.max(np.abs(H)), scale ** 2)
    return g, o


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [1, 2, 3, 37, 96, 161])
def test_random_hermitian_matches_the_oracle(cplx, n):
    """Random indefinite H: mixed 1x1 and 2x2 pivots (a Gaussian Hermitian
    matrix takes 2x2 pivots at a good share of the steps)."""
    rng = np.random.default_rng(1000 + 7 * n + cplx)
    H = _herm(n, cplx, rng)
    g, o = _check_against_oracle(H)
    if n >= 37:
        assert 2 in o["block_sizes"] and 1 in o["block_sizes"]


@pytest.mark.parametrize("cplx", [False, True])
def test_definite_and_graded_inputs(cplx):
    """A definite H (only 1x1 pivots: diagonal pivoting, pivoted Cholesky) and
    a strongly graded indefinite one (entries over 12 orders of magnitude)."""
    rng = np.random.default_rng(77 + cplx)
    n = 64
    X = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    Hd = X @ X.conj().T + n * np.eye(n)
    Hd = (Hd + Hd.conj().T) / 2
    g, o = _check_against_oracle(-Hd)
    assert o["block_sizes"] == [1] * n and np.all(g["J"] == -1)
    D = np.logspace(0, -6, n)
    Hg = D[:, None] * _herm(n, cplx, rng) * D[None, :]
    _check_against_oracle((Hg + Hg.conj().T) / 2)


@pytest.mark.parametrize("cplx", [False, True])
def test_special_cases(cplx):
    """Zero diagonal (every pivot 2x2), a diagonal matrix (1x1 pivots in the
    order of decreasing modulus, ties to the lower index), and the zero matrix
    (rank 0)."""
    rng = np.random.default_rng(5 + cplx)
    n = 40
    H = _herm(n, cplx, rng)
    np.fill_diagonal(H, 0.0)
    g, o = _check_against_oracle(H)
    assert o["block_sizes"][0] == 2
    d = np.array([3.0, -5.0, 5.0, 0.5, -3.0, 1.0, 2.0, -0.25])
    H = np.diag(d).astype(np.complex128 if cplx else np.float64)
    g, o = _check_against_oracle(H)
    assert list(g["perm"]) == [1, 2, 0, 4, 6, 5, 3, 7]
    assert list(g["J"]) == [-1, 1, 1, -1, 1, 1, 1, -1]
    Z = np.zeros((9, 9), dtype=H.dtype)
    g = _factor_gpu(Z)
    assert g["rank"] == 0


@pytest.mark.parametrize("cplx", [False, True])
def test_singular_h_rank_and_inertia(cplx):
    """H of rank r < n with p positive and r - p negative eigenvalues: the
    factor has r columns, J has p positive signs (Sylvester), and the rank
    equals the oracle's."""
    rng = np.random.default_rng(31 + cplx)
    n, r, p = 72, 50, 29
    lam = np.concatenate([rng.uniform(0.5, 2.0, p), -rng.uniform(0.5, 2.0, r - p), np.zeros(n - r)])
    H = _known(n, cplx, rng, lam)
    g, o = _check_against_oracle(H, rank_tol=1e-10)
    assert g["rank"] == r and int(np.sum(g["J"] > 0)) == p


@pytest.mark.parametrize("cplx", [False, True])
def test_eigenvalues_of_h_through_the_whole_method(cplx):
    """H with prescribed eigenvalues over six orders of magnitude: front end on
    the GPU, one-sided J-Jacobi of (G, J) on the GPU, lambda_i = J_ii
    ||g~_i||^2; compared with the oracle's whole method and with the
    prescribed values."""
    rng = np.random.default_rng(400 + cplx)
    n = 80
    mags = np.logspace(0, -6, n)
    lam = mags * np.where(rng.random(n) < 0.4, -1.0, 1.0)
    H = _known(n, cplx, rng, lam)
    g = _factor_gpu(H)
    assert g["rank"] == n
    res = solve_gpu(g["G"], g["J"].astype(np.int8))
    assert res["info"]["status"] == 0
    ref = frontend.eigh_via_jjacobi(H)
    assert max_rel_err(res["lam"], ref["lam"]) <= 1e-9
    assert max_rel_err(res["lam"], lam) <= 1e-9
