"""CPU oracle for the front end of the one-sided J-Jacobi method: the
Hermitian indefinite factorization H -> (G, J) of Sec. 2.2, (2.5), and the
zero-eigenvalue completion of a singular H described after (2.11).

TEST INFRASTRUCTURE ONLY, under the same contract as the rest of this package:
only the tests, the smoke check and the benchmark's CPU-baseline leg import
it, and the product library neither imports nor calls it.

Contents
  bunch_parlett(H)     P H P^T = M D M^* with complete (Bunch-Parlett)
                       pivoting: M unit lower trapezoidal (n x r), D block
                       diagonal with Hermitian blocks of order 1 or 2.
  factor_gj(H)         G (n x r, rows in H's order) and J (r signs) with
                       H = G J G^*: each block of D diagonalized and the
                       columns of M scaled by |delta|^(1/2) (2.5).
  zero_eigenvectors(U) an orthonormal basis of the orthogonal complement of
                       range(U), from a full QR factorization.
  eigh_via_jjacobi(H)  the whole method on H: factor, one-sided J-Jacobi
                       (the plain oracle), eigenpairs, completion.

Readings where the paper is silent (it refers the factorization variant to its
references):
  * pivoting is the classical complete pivoting of Bunch and Parlett with
    alpha = (1 + sqrt 17) / 8: with mu0 the largest modulus in the Schur
    complement and mu1 the largest modulus on its diagonal, a 1x1 pivot at
    argmax |s_ii| when mu1 >= alpha mu0, else the 2x2 pivot on the
    off-diagonal entry of modulus mu0;
  * the rank is the number of columns eliminated before mu0 falls to
    rank_tol times its initial value (default 16 n eps); the rest of the
    Schur complement is dropped, which gives the n x r factor of full column
    rank that the paper describes for a singular H;
  * the Schur complement is formed from its lower triangle and mirrored,
    with a real diagonal, so that it stays exactly Hermitian;
  * a 2x2 block is diagonalized by an eigendecomposition Q diag(delta) Q^*
    (LAPACK's Hermitian eigensolver on the 2x2 block), giving the columns
    M_b Q |delta|^(1/2) with signs sign(delta); the pivot rule makes the two
    deltas of opposite sign.

Pinned by tests/test_oracle_frontend.py.
"""
from __future__ import annotations

from typing import Dict, List, Optional

import numpy as np

from . import eigenpairs, solve_plain

ALPHA_BUNCH_PARLETT = (1.0 + np.sqrt(17.0)) / 8.0
EPS = 2.0 ** -53


def bunch_parlett(H: np.ndarray, rank_tol: Optional[float] = None,
                  mutation: int = 0) -> Dict[str, object]:
    """P H P^T = M D M^* by symmetric Gaussian elimination with complete
    pivoting (Sec. 2.2). Returns perm (P H P^T = H[perm][:, perm]), M (n x r,
    unit lower trapezoidal in the permuted order), the list of diagonal
    blocks of D and their offsets, and r.

    mutation 1 plants a mistake for the tests: the Schur complement update
    uses C E^{-1} C^T instead of C E^{-1} C^* (wrong for complex H)."""
    A = np.array(H, dtype=np.complex128 if np.iscomplexobj(H) else np.float64, copy=True)
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("H must be square")
    if not np.allclose(A, A.conj().T, rtol=0, atol=0):
        raise ValueError("H must be Hermitian")
    tol = 16 * n * EPS if rank_tol is None else rank_tol
    perm = np.arange(n)
    M = np.zeros_like(A)
    blocks: List[np.ndarray] = []
    offsets: List[int] = []
    mu0_init = np.max(np.abs(A)) if n else 0.0
    k = 0
    while k < n:
        S = A[k:, k:]
        absS = np.abs(S)
        mu0 = absS.max()
        if mu0 == 0.0 or mu0 <= tol * mu0_init:
            break
        diag = np.abs(np.diag(S))  # real: the diagonal of a Hermitian matrix
        mu1 = diag.max()
        if mu1 >= ALPHA_BUNCH_PARLETT * mu0 or k == n - 1:
            piv = [k + int(np.argmax(diag))]
        else:
            off = absS.copy()
            np.fill_diagonal(off, -1.0)
            i, j = np.unravel_index(int(np.argmax(off)), off.shape)
            piv = [k + min(i, j), k + max(i, j)]
        s = len(piv)
        # symmetric interchanges bring the pivot rows/columns to k .. k+s-1
        # (a 2x2 pivot has piv[0] < piv[1], so the first interchange never
        # moves the second pivot)
        for t, p in enumerate(piv):
            dst = k + t
            if p != dst:
                A[[dst, p], :] = A[[p, dst], :]
                A[:, [dst, p]] = A[:, [p, dst]]
                M[[dst, p], :] = M[[p, dst], :]
                perm[[dst, p]] = perm[[p, dst]]
        E = A[k:k + s, k:k + s].copy()
        C = A[k + s:, k:k + s].copy()
        L = np.linalg.solve(E.T, C.T).T  # L = C E^{-1}
        M[k:k + s, k:k + s] = np.eye(s)
        M[k + s:, k:k + s] = L
        CE = C.T if mutation == 1 else C.conj().T
        T = A[k + s:, k + s:] - L @ CE
        # the Schur complement is Hermitian: keep its lower triangle, mirror
        # it, and keep the diagonal real (rounding would otherwise drift it
        # away from symmetry, and M D M^* would no longer reproduce H)
        T = np.tril(T, -1) + np.tril(T, -1).conj().T + np.diag(np.real(np.diag(T)))
        A[k + s:, k + s:] = T
        A[k + s:, k:k + s] = 0
        A[k:k + s, k + s:] = 0
        blocks.append(E)
        offsets.append(k)
        k += s
    r = k
    return dict(perm=perm, M=M[:, :r], blocks=blocks, offsets=offsets, rank=r)


def factor_gj(H: np.ndarray, rank_tol: Optional[float] = None,
              mutation: int = 0) -> Dict[str, object]:
    """G and J with H = G J G^* (2.5): the blocks of D diagonalized, the
    columns of M scaled by |delta|^(1/2), and the rows returned to H's order.
    G is n x r of full column rank; J holds r signs in elimination order."""
    f = bunch_parlett(H, rank_tol=rank_tol, mutation=mutation)
    M, perm = f["M"], f["perm"]
    n, r = M.shape
    Gp = np.zeros_like(M)
    J = np.zeros(r, dtype=np.int8)
    for E, k in zip(f["blocks"], f["offsets"]):
        s = E.shape[0]
        if s == 1:
            d = float(np.real(E[0, 0]))
            Gp[:, k] = M[:, k] * np.sqrt(abs(d))
            J[k] = 1 if d > 0 else -1
        else:
            delta, Q = np.linalg.eigh(E)
            Gp[:, k:k + 2] = (M[:, k:k + 2] @ Q) * np.sqrt(np.abs(delta))
            J[k:k + 2] = np.where(delta > 0, 1, -1)
    G = np.zeros_like(Gp)
    G[perm, :] = Gp
    return dict(G=G, J=J, perm=perm, rank=r, block_sizes=[E.shape[0] for E in f["blocks"]],
                Gp=Gp)


def zero_eigenvectors(U: np.ndarray) -> np.ndarray:
    """Orthonormal basis of the orthogonal complement of range(U) (n x r,
    orthonormal columns): the trailing n - r columns of Q in the full QR
    factorization U = Q R (the completion after (2.11))."""
    n, r = U.shape
    Q, _ = np.linalg.qr(U, mode="complete")
    return Q[:, r:]


def eigh_via_jjacobi(H: np.ndarray, rank_tol: Optional[float] = None,
                     tol: Optional[float] = None) -> Dict[str, object]:
    """Eigenvalues and eigenvectors of a Hermitian H by the paper's method:
    factor H = G J G^* (Sec. 2.2), orthogonalize the columns of G by the
    one-sided J-Jacobi method (Alg. 3.2), read off lambda_i = J_ii ||g~_i||^2
    and u_i = g~_i / ||g~_i|| (2.11), and complete a singular H's eigenvectors
    for the zero eigenvalue."""
    f = factor_gj(H, rank_tol=rank_tol)
    G, J = f["G"], f["J"]
    n, r = G.shape
    kw = {} if tol is None else dict(tol=tol)
    if r == 0:
        return dict(lam=np.zeros(n), U=np.eye(n, dtype=G.dtype), rank=0, status=0, sweeps=0)
    res = solve_plain(G, J, **kw)
    lam, U = eigenpairs(res["Gt"], J)
    lam = np.asarray(lam, dtype=np.float64)
    U = np.asarray(U)
    if r < n:
        Z = zero_eigenvectors(U)
        lam = np.concatenate([lam, np.zeros(n - r)])
        U = np.concatenate([U, Z.astype(U.dtype)], axis=1)
    return dict(lam=lam, U=U, rank=r, status=res["status"], sweeps=res["sweeps"])
