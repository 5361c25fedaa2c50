"""GPU parity of the blocked full-block path (Gram, inner solve, update, whole
solve) against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import (U64, eig_rel_tol, max_rel_err, orth_residual, pivot_rel_tol,
                         reconstruction_residual)
from tests.gpu_util import col_rel_err, dtype_of, from_dev, require_gpu, solve_gpu, to_dev

pytestmark = pytest.mark.gpu

GEMMS = [0, 1]  # JJ_GEMM_FP64, JJ_GEMM_OZAKI_FP16


def _pairs_for(n, sizes_pairs):
    """Pair descriptors {off_i, n_i, off_j, n_j} for a list of ((i0, ni), (j0, nj))."""
    return np.array([[a, na, b, nb] for (a, na), (b, nb) in sizes_pairs], dtype=np.int32)


def _random_pairs(n, rng, count, nb_lo, nb_hi):
    """Disjoint random block pairs inside n columns (ragged widths)."""
    cols = rng.permutation(n // nb_hi)  # block slots of width nb_hi
    out = []
    for q in range(count):
        i, j = cols[2 * q], cols[2 * q + 1]
        ni = int(rng.integers(nb_lo, nb_hi + 1))
        nj = int(rng.integers(nb_lo, nb_hi + 1))
        out.append(((i * nb_hi, ni), (j * nb_hi, nj)))
    return _pairs_for(n, out)


def _pivot(G, pd):
    a, na, b, nb = pd
    return np.concatenate([G[:, a:a + na], G[:, b:b + nb]], axis=1)


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("gemm", GEMMS)
@pytest.mark.parametrize("m", [300, 1111])
def test_gram_matches_oracle(cplx, gemm, m):
    jj = require_gpu()
    import torch
    rng = np.random.default_rng(m + 7 * cplx + gemm)
    n = 160
    G = rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cplx else 0)
    G *= 10.0 ** rng.uniform(-4, 4, size=(m, 1))  # graded rows
    G = np.asfortranarray(G)
    hi = 16 if (gemm == 1 and cplx) else 20  # the digit form takes real widths <= 64
    pairs = _random_pairs(n, rng, 4, 9, hi)
    kmax = 2 * hi
    Gd = to_dev(G)
    pd = torch.from_numpy(pairs).cuda()
    A = torch.zeros(len(pairs) * kmax * kmax * (2 if cplx else 1), dtype=torch.float64,
                    device="cuda")
    jj.jjk_gram(dtype_of(G), gemm, Gd, Gd.stride(1), m, pd, len(pairs), A, kmax)
    torch.cuda.synchronize()
    Ah = A.cpu().numpy()
    if cplx:
        Ah = Ah.view(np.complex128)
    Ah = Ah.reshape(len(pairs), kmax, kmax).transpose(0, 2, 1)  # column-major blocks
    for q, p in enumerate(pairs):
        k = p[1] + p[3]
        ref = oracle.gram(_pivot(G, p))
        d = np.sqrt(np.abs(np.diag(ref)).real)
        err = np.abs(Ah[q, :k, :k] - ref) / np.outer(d, d)
        assert err.max() <= 64 * U64 * np.sqrt(m), (q, err.max())


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("gemm", GEMMS)
def test_update_matches_oracle(cplx, gemm):
    jj = require_gpu()
    import torch
    rng = np.random.default_rng(3 + cplx + 10 * gemm)
    hi = 16 if (gemm == 1 and cplx) else 24  # the digit form takes real widths <= 64
    m, n, kmax = 517, 120, 2 * hi
    G = rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cplx else 0)
    G *= 10.0 ** rng.uniform(-3, 3, size=(m, 1))
    G = np.asfortranarray(G)
    pairs = _random_pairs(n, rng, 2, 11, hi)
    Ws = []
    Wbuf = np.zeros((len(pairs), kmax, kmax), dtype=G.dtype)
    for q, p in enumerate(pairs):
        k = p[1] + p[3]
        W = rng.standard_normal((k, k)) + (1j * rng.standard_normal((k, k)) if cplx else 0)
        W *= 10.0 ** rng.uniform(-2, 2, size=(1, k))
        Ws.append(W)
        Wbuf[q, :k, :k] = W
    Wd = torch.from_numpy(np.ascontiguousarray(Wbuf.transpose(0, 2, 1))).cuda()
    Wd = torch.view_as_real(Wd).reshape(-1) if cplx else Wd.reshape(-1)
    Gs = to_dev(G)
    Gd = to_dev(np.zeros_like(G))
    pd = torch.from_numpy(pairs).cuda()
    jj.jjk_update(dtype_of(G), gemm, Gs, Gd, Gs.stride(1), m, pd, len(pairs), Wd, kmax)
    torch.cuda.synchronize()
    out = from_dev(Gd)
    for q, p in enumerate(pairs):
        ref = oracle.update(_pivot(G, p), Ws[q])
        got = _pivot(out, p)
        # error relative to |G_P| |W| row by row (FP64 GEMM error model)
        bound = np.abs(_pivot(G, p)) @ np.abs(Ws[q])
        assert np.max(np.abs(got - ref) / bound) <= 64 * U64 * np.sqrt(p[1] + p[3])


@pytest.mark.parametrize("cplx", [True, False])
def test_inner_matches_oracle(cplx):
    """Cholesky + inner J-Jacobi with W accumulated: R~ = R W with R the oracle's
    Cholesky factor, W J-unitary, columns of R~ orthogonal, and the pair's
    eigenvalues J_c ||r~_c||^2 equal the oracle's inner solve."""
    jj = require_gpu()
    import torch
    P = synth.make_workload("plain_c128_n128" if cplx else "blocked_f64_n2048_b32", n=96)
    rng = np.random.default_rng(2)
    pairs = _pairs_for(96, [((0, 20), (50, 21)), ((30, 19), (71, 20))])
    kmax = 42
    E = 2 if cplx else 1
    A = np.zeros((len(pairs), kmax, kmax), dtype=P.G.dtype)
    Rs, JPs = [], []
    for q, p in enumerate(pairs):
        GP = _pivot(P.G, p)
        AP = oracle.gram(GP)
        k = p[1] + p[3]
        A[q, :k, :k] = AP
        Rs.append(oracle.cholesky_upper(AP))
        JPs.append(np.concatenate([P.J[p[0]:p[0] + p[1]], P.J[p[2]:p[2] + p[3]]]))
    Ad = torch.from_numpy(np.ascontiguousarray(A.transpose(0, 2, 1))).cuda()
    Ad = (torch.view_as_real(Ad) if cplx else Ad).reshape(-1).contiguous()
    Wd = torch.zeros_like(Ad)
    Jd = torch.from_numpy(P.J.astype(np.int8)).cuda()
    cnt = torch.zeros(8, dtype=torch.int64, device="cuda")
    pd = torch.from_numpy(pairs).cuda()
    jj.jjk_inner(dtype_of(P.G), Ad, Wd, kmax, pd, len(pairs), Jd, 0.0, 30, 0, cnt)
    torch.cuda.synchronize()
    assert int(cnt[2]) == 0
    Rt = Ad.cpu().numpy()
    Wt = Wd.cpu().numpy()
    if cplx:
        Rt, Wt = Rt.view(np.complex128), Wt.view(np.complex128)
    Rt = Rt.reshape(len(pairs), kmax, kmax).transpose(0, 2, 1)
    Wt = Wt.reshape(len(pairs), kmax, kmax).transpose(0, 2, 1)
    for q, p in enumerate(pairs):
        k = p[1] + p[3]
        R, W, JP = Rs[q], Wt[q, :k, :k], JPs[q]
        Jm = np.diag(JP.astype(np.float64))
        wmax = np.abs(W).max()
        assert np.abs(W.conj().T @ Jm @ W - Jm).max() <= 1e4 * U64 * wmax ** 2
        # The GPU's Cholesky factor, recovered as R~ W^{-1} = R~ J W^* J, is upper
        # triangular and reproduces A_P to the Cholesky backward error (its forward
        # error against LAPACK's factor grows with cond(A_P), so it is not compared).
        Rg = Rt[q, :k, :k] @ (Jm @ W.conj().T @ Jm)
        AP = R.conj().T @ R
        dd = np.sqrt(np.abs(np.diag(AP)))
        scale = np.abs(Rt[q, :k, :k]).max() * wmax
        assert np.abs(np.tril(Rg, -1)).max() <= 1e4 * U64 * scale
        assert np.max(np.abs(Rg.conj().T @ Rg - AP) / np.outer(dd, dd)) <= 1e4 * U64 * wmax ** 2
        lam_gpu = JP * np.linalg.norm(Rt[q, :k, :k], axis=0) ** 2
        ref = oracle.inner_solve(R, JP)
        assert max_rel_err(lam_gpu, ref["lam"]) <= pivot_rel_tol(R)
        U = Rt[q, :k, :k] / np.linalg.norm(Rt[q, :k, :k], axis=0)
        assert orth_residual(U) <= 8 * oracle.TOL_DEFAULT


@pytest.mark.parametrize("gemm", GEMMS)
@pytest.mark.parametrize("order", [0, 1])
def test_blocked_real_matches_oracle(gemm, order):
    require_gpu()
    P = synth.make_workload("blocked_f64_n2048_b32", n=256)
    ref = oracle.solve_plain(P.G, P.J)
    got = solve_gpu(P.G, P.J, block_width=32, gemm=gemm, order=order, want_U=True)
    tol = eig_rel_tol(P.G)
    assert got["info"]["status"] == 0
    assert got["info"]["nbl"] == 8
    assert max_rel_err(got["lam"], ref["lam"]) <= tol
    assert max_rel_err(got["lam"], P.lam_exact) <= tol
    assert orth_residual(got["U"]) <= 8 * oracle.TOL_DEFAULT
    assert reconstruction_residual(P.G, P.J, got["lam"], got["U"]) <= 1e-12


@pytest.mark.parametrize("gemm", GEMMS)
def test_blocked_complex_ragged(gemm):
    """Complex, n not a multiple of 2b (uniform partition with ragged blocks)."""
    require_gpu()
    P = synth.make_workload("plain_c128_n128", n=150)
    ref = oracle.solve_plain(P.G, P.J)
    got = solve_gpu(P.G, P.J, block_width=11, gemm=gemm)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= eig_rel_tol(P.G)
    assert max_rel_err(got["lam"], P.lam_exact) <= eig_rel_tol(P.G)


@pytest.mark.parametrize("gemm", [0, 1, 2])
def test_blocked_graded_complex(gemm):
    """Graded G = D1 B D2 (the graded complex recipe at n = 192): the published
    bound for the graded case, 1e-10 relative to the FP64 oracle. (The scaled
    condition of G is far above 1e4 here; the FP64 oracle and its long-double
    variant agree to ~1e-12 on these inputs, so the bound is meaningful.)"""
    require_gpu()
    P = synth.make_workload("graded_c128_n4096_b64", n=192)
    ref = oracle.solve_plain(P.G, P.J)
    got = solve_gpu(P.G, P.J, block_width=16, gemm=gemm)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= 1e-10


@pytest.mark.parametrize("gemm", GEMMS)
def test_one_parallel_step_through_building_blocks(gemm):
    """One parallel step (Gram -> inner -> update for every pair of step 0)
    through the kernel entry points: every pivot pair is diagonalized, and the
    sorted J_c ||g_c||^2 over its columns (the pair pencil's eigenvalues, which
    are unique) equal those after the oracle's first step."""
    jj = require_gpu()
    import torch
    P = synth.make_workload("plain_c128_n128", n=64)
    b = 8
    ref = oracle.solve_blocked(P.G, P.J, b, max_steps=1)
    nbl, sizes = ref["nbl"], ref["sizes"]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    tab = jj.jjacobi_schedule(nbl, 0, 1)
    pairs = np.array([[offs[i], sizes[i], offs[j], sizes[j]] for i, j in tab[0]], dtype=np.int32)
    kmax = 2 * max(sizes)
    Gs = to_dev(P.G)
    Gd = to_dev(np.zeros_like(P.G))
    pd = torch.from_numpy(pairs).cuda()
    A = torch.zeros(len(pairs) * kmax * kmax * 2, dtype=torch.float64, device="cuda")
    W = torch.zeros_like(A)
    Jd = torch.from_numpy(P.J.astype(np.int8)).cuda()
    cnt = torch.zeros(8, dtype=torch.int64, device="cuda")
    jj.jjk_gram(jj.JJ_C128, gemm, Gs, Gs.stride(1), P.m, pd, len(pairs), A, kmax)
    jj.jjk_inner(jj.JJ_C128, A, W, kmax, pd, len(pairs), Jd, 0.0, 30, 0, cnt)
    jj.jjk_update(jj.JJ_C128, gemm, Gs, Gd, Gs.stride(1), P.m, pd, len(pairs), W, kmax)
    torch.cuda.synchronize()
    assert int(cnt[2]) == 0 and int(cnt[0]) > 0
    out = from_dev(Gd)
    lam_ref = P.J * np.linalg.norm(ref["Gt"], axis=0) ** 2
    lam_gpu = P.J * np.linalg.norm(out, axis=0) ** 2
    for p in pairs:
        cols = np.r_[p[0]:p[0] + p[1], p[2]:p[2] + p[3]]
        R0 = oracle.cholesky_upper(oracle.gram(P.G[:, cols]))
        assert max_rel_err(lam_gpu[cols], lam_ref[cols]) <= pivot_rel_tol(R0)
        # After one step the pivot columns are orthogonal up to the Gram and
        # Cholesky errors carried through W_P, as in the oracle's own step.
        U = out[:, cols] / np.linalg.norm(out[:, cols], axis=0)
        Ur = ref["Gt"][:, cols] / np.linalg.norm(ref["Gt"][:, cols], axis=0)
        assert orth_residual(U) <= max(8 * oracle.TOL_DEFAULT, 10 * orth_residual(Ur))


@pytest.mark.parametrize("gemm", [0, 1])
def test_autotuned_block_width(gemm):
    """block_width = JJ_BLOCK_AUTO: the first solve times one sweep per candidate
    width and keeps the fastest; the result is the blocked solve with that width."""
    jj = require_gpu()
    import torch

    P = synth.make_workload("plain_c128_n128", n=160)
    m, n = P.G.shape
    with jj.Handle(m, n, jj.JJ_C128, block_width=jj.JJ_BLOCK_AUTO, gemm=gemm) as h:
        infos = []
        for _ in range(2):
            Gd = to_dev(P.G)
            infos.append(h.jjacobi_solve(Gd, Gd.stride(1), P.J).as_dict())
            lam = torch.empty(n, dtype=torch.float64, device="cuda")
            h.jjacobi_extract(lam)
            assert max_rel_err(lam.cpu().numpy(), P.lam_exact) <= eig_rel_tol(P.G)
    b = infos[0]["block_width"]
    assert b in ([8, 16] if gemm == 1 else [8, 16, 32])
    assert infos[1]["block_width"] == b
    fixed = solve_gpu(P.G, P.J, block_width=b, gemm=gemm)
    assert fixed["info"]["sweeps"] == infos[1]["sweeps"]


@pytest.mark.parametrize("gemm", [0, 1, 2])
def test_block_oriented_real_matches_oracle(gemm):
    """Block-oriented strategy (B, Sec. 5.3 / Alg. 3.4): one full pass over each
    pivot in the first step of a sweep, one pass over the off-diagonal block in
    the others."""
    require_gpu()
    from paper_1008_4166_gb300 import jjacobi as jj

    P = synth.make_workload("blocked_f64_n2048_b32", n=256)
    ref = oracle.solve_plain(P.G, P.J)
    got = solve_gpu(P.G, P.J, block_width=32, gemm=gemm, want_U=True,
                    block_strategy=jj.JJ_BLOCK_ORIENTED)
    tol = eig_rel_tol(P.G)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= tol
    assert max_rel_err(got["lam"], P.lam_exact) <= tol
    assert orth_residual(got["U"]) <= 8 * oracle.TOL_DEFAULT
    assert reconstruction_residual(P.G, P.J, got["lam"], got["U"]) <= 1e-12


@pytest.mark.parametrize("order", [0, 1])
def test_block_oriented_complex_ragged_and_graded(order):
    """Unequal block sizes (150 columns, b = 11: off-diagonal blocks of 10 x 11)
    and the graded recipe held to 1e-10 (hybrid and all-digit forms)."""
    require_gpu()
    from paper_1008_4166_gb300 import jjacobi as jj

    P = synth.make_workload("plain_c128_n128", n=150)
    ref = oracle.solve_plain(P.G, P.J)
    got = solve_gpu(P.G, P.J, block_width=11, gemm=0, order=order,
                    block_strategy=jj.JJ_BLOCK_ORIENTED)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= eig_rel_tol(P.G)
    Pg = synth.make_workload("graded_c128_n4096_b64", n=192)
    refg = oracle.solve_plain(Pg.G, Pg.J)
    for gemm in (2, 1):  # hybrid, all-digit
        gg = solve_gpu(Pg.G, Pg.J, block_width=16, gemm=gemm, order=order,
                       block_strategy=jj.JJ_BLOCK_ORIENTED)
        assert gg["info"]["status"] == 0
        assert max_rel_err(gg["lam"], refg["lam"]) <= 1e-10, gemm


def test_block_oriented_rejects_pivots_beyond_shared_memory():
    """Single passes run in the shared-memory inner kernel: a two-level
    block-oriented solve with 256-column pivots is refused (the three-level
    form takes such pivots)."""
    jj = require_gpu()
    with pytest.raises(jj.JJError):
        jj.Handle(1024, 1024, jj.JJ_F64, block_width=128, block_strategy=jj.JJ_BLOCK_ORIENTED)
