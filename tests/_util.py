"""Shared helpers for the tests: tolerances and error measures (no solver arithmetic)."""
import numpy as np

U64 = 2.0 ** -53  # unit roundoff of float64


def kappa_scaled(G: np.ndarray) -> float:
    """Condition of G with unit-norm columns, kappa(G diag(1/||g_i||)).

    One-sided J-Jacobi is accurate relative to this quantity (the scaled
    condition of the relative perturbation theory cited in Sec. 1)."""
    Gs = G / np.linalg.norm(G, axis=0)[None, :]
    s = np.linalg.svd(Gs, compute_uv=False)
    return float(s[0] / s[-1])


def eig_rel_tol(G: np.ndarray, floor: float = 1e-12, factor: float = 4.0) -> float:
    """Relative eigenvalue tolerance: max(floor, factor * u * kappa_scaled(G)).

    The floor is the published target for well-conditioned inputs; above a
    scaled condition of ~2e3 the first-order bound u * kappa dominates, and no
    float64 method can be held to less."""
    return max(floor, factor * U64 * kappa_scaled(G))


def max_rel_err(a, b) -> float:
    a = np.sort(np.asarray(a, dtype=np.float64))
    b = np.sort(np.asarray(b, dtype=np.float64))
    return float(np.max(np.abs(a - b) / np.abs(b)))


def orth_residual(U: np.ndarray) -> float:
    """max_{i != j} |u_i^* u_j| for unit columns (orthonormality of U~, (2.10))."""
    U = np.asarray(U).astype(np.complex128 if np.iscomplexobj(U) else np.float64)
    M = U.conj().T @ U
    return float(np.max(np.abs(M - np.diag(np.diag(M)))))


def reconstruction_residual(G: np.ndarray, J, lam, U) -> float:
    """||G J G^* - U diag(lam) U^*||_F / ||G||_F^2 (the HSVD identity, Sec. 2.3)."""
    G = np.asarray(G)
    Jd = np.asarray(J, dtype=np.float64)
    H = (G * Jd[None, :]) @ G.conj().T
    U = np.asarray(U).astype(G.dtype)
    Hr = (U * np.asarray(lam, dtype=np.float64)[None, :]) @ U.conj().T
    return float(np.linalg.norm(H - Hr) / np.linalg.norm(G) ** 2)


def pivot_rel_tol(R, k=None, factor: float = 8.0) -> float:
    """Tolerance for eigenvalues of one pivot pencil (R^* R, J_P) when the two
    sides start from Cholesky factors that differ by the Cholesky backward
    error |E_ij| <= c k u sqrt(a_ii a_jj): that perturbation moves the pencil's
    eigenvalues by up to ~ k u kappa(A_s) with kappa(A_s) = kappa(R_s)^2."""
    k = R.shape[1] if k is None else k
    ks = kappa_scaled(R)
    return max(eig_rel_tol(R), factor * k * U64 * ks * ks)
