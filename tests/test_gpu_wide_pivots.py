"""Digit-product Gram (3.6) and update (2.9) for pivots wider than one
64-position tile of the real form (complex pivots of more than 32 columns,
real ones of more than 64, up to 256 positions): the building blocks against
the oracle's Gram and the exact (long double) product, ragged tiles included,
and whole solves whose outer contractions take this path."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import U64, eig_rel_tol, max_rel_err
from tests.gpu_util import dtype_of, from_dev, require_gpu, solve_gpu, to_dev

pytestmark = pytest.mark.gpu


def _pivot(G, p):
    a, na, b, nb = p
    return np.concatenate([G[:, a:a + na], G[:, b:b + nb]], axis=1)


def _pairs(sizes, rng):
    offs = np.concatenate([[0], np.cumsum(sizes)])
    perm = rng.permutation(len(sizes))
    return np.array([[offs[perm[2 * q]], sizes[perm[2 * q]], offs[perm[2 * q + 1]],
                      sizes[perm[2 * q + 1]]] for q in range(len(sizes) // 2)], dtype=np.int32)


@pytest.mark.parametrize("cplx", [True, False])
def test_wide_gram_matches_oracle(cplx):
    """Pivots of 2 to 4 tiles per side with ragged last tiles (complex blocks
    of 17..64 columns, real ones of 33..128), graded rows over 8 orders of
    magnitude, 300 rows (ragged 128-row accumulations)."""
    jj = require_gpu()
    import torch
    rng = np.random.default_rng(71 + cplx)
    m = 300
    sizes = rng.integers(17, 65, size=8) if cplx else rng.integers(33, 129, size=8)
    sizes[0] = 64 if cplx else 128  # one pivot at the full 256 positions
    sizes[1] = 64 if cplx else 128
    n = int(np.sum(sizes))
    G = rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cplx else 0)
    G = np.asfortranarray(G * 10.0 ** rng.uniform(-4, 4, size=(m, 1)))
    pairs = _pairs(sizes, rng)
    pairs[0] = [0, sizes[0], sizes[0], sizes[1]]
    kmax = int(max(p[1] + p[3] for p in pairs))
    Gd = to_dev(G)
    pd = torch.from_numpy(pairs).cuda()
    A = torch.zeros(len(pairs) * kmax * kmax * (2 if cplx else 1), dtype=torch.float64, device="cuda")
    jj.jjk_gram(dtype_of(G), jj.JJ_GEMM_OZAKI_FP16, Gd, Gd.stride(1), m, pd, len(pairs), A, kmax)
    torch.cuda.synchronize()
    Ah = A.cpu().numpy()
    if cplx:
        Ah = Ah.view(np.complex128)
    Ah = Ah.reshape(len(pairs), kmax, kmax).transpose(0, 2, 1)
    for q, p in enumerate(pairs):
        k = p[1] + p[3]
        ref = oracle.gram(_pivot(G, p))
        d = np.sqrt(np.abs(np.diag(ref)).real)
        err = np.abs(Ah[q, :k, :k] - ref) / np.outer(d, d)
        assert err.max() <= 64 * U64 * np.sqrt(m), (q, k, err.max())
        # the lower tiles are read as the transposes of the upper ones (the
        # integer sums are exact): the real part is exactly symmetric
        assert np.array_equal(Ah[q, :k, :k].real, Ah[q, :k, :k].real.T)


def _update(jj, G, pairs, Ws, kmax, inplace):
    import torch
    Gs = to_dev(G)
    Gd = Gs if inplace else to_dev(np.zeros_like(G))
    Wbuf = np.zeros((len(pairs), kmax, kmax), dtype=G.dtype)
    for q, W in enumerate(Ws):
        Wbuf[q, :W.shape[0], :W.shape[1]] = W
    Wd = torch.from_numpy(np.ascontiguousarray(Wbuf.transpose(0, 2, 1))).cuda()
    Wd = torch.view_as_real(Wd).reshape(-1) if np.iscomplexobj(G) else Wd.reshape(-1)
    pd = torch.from_numpy(np.asarray(pairs, dtype=np.int32)).cuda()
    jj.jjk_update(dtype_of(G), jj.JJ_GEMM_OZAKI_FP16, Gs, Gd, Gs.stride(1), G.shape[0], pd,
                  len(pairs), Wd, kmax)
    torch.cuda.synchronize()
    return from_dev(Gd)


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("inplace", [True, False])
def test_wide_update_within_fp64_entry_bound(cplx, inplace):
    """[G_i G_j] W_P for pivots of 2, 3 and 4 tiles per side (with ragged
    tiles), J-unitary-like W = I + graded perturbation, graded rows, 300 rows:
    every sampled entry within twice FP64's own bound
    u (|x_lj| + sum_a |x_la| |w_aj - delta_aj|) of the exact product (long
    double); columns outside every pair unchanged."""
    jj = require_gpu()
    rng = np.random.default_rng(5 + cplx + 2 * inplace)
    m = 300
    ks = [128, 72, 40, 100] if cplx else [256, 200, 100, 130]  # pivot widths (columns)
    sizes = []
    for k in ks:
        sizes += [k // 2, k - k // 2]
    sizes += [7]  # a column block outside every pair
    offs = np.concatenate([[0], np.cumsum(sizes)])
    n = int(offs[-1])
    G = rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cplx else 0)
    G = np.asfortranarray(G * 10.0 ** rng.uniform(-3, 3, size=(m, 1)))
    pairs = [[offs[2 * q], sizes[2 * q], offs[2 * q + 1], sizes[2 * q + 1]] for q in range(len(ks))]
    kmax = max(ks)
    Ws = []
    for k in ks:
        E = rng.standard_normal((k, k)) + (1j * rng.standard_normal((k, k)) if cplx else 0)
        Ws.append(np.eye(k) + 1e-2 * E * 10.0 ** rng.uniform(-2, 2, size=(1, k)))
    out = _update(jj, G, pairs, Ws, kmax, inplace)
    L = np.longdouble
    rows = np.r_[0:40, 250:300]  # a sample of rows (long double is slow), both ragged ends
    for q, p in enumerate(pairs):
        X = _pivot(G, p)[rows]
        W = Ws[q]
        if cplx:
            Xr = np.concatenate([X.real, X.imag], axis=1).astype(L)
            W2 = np.block([[W.real, W.imag], [-W.imag, W.real]]).astype(L)
        else:
            Xr, W2 = X.astype(L), W.astype(L)
        exact = Xr @ W2
        D = np.abs(W2 - np.eye(W2.shape[0], dtype=L))
        bound = (np.abs(Xr) @ D + np.abs(Xr)) * U64
        Y = _pivot(out, p)[rows]
        got = (np.concatenate([Y.real, Y.imag], axis=1) if cplx else Y).astype(L)
        ratio = float(np.max(np.abs(got - exact) / np.maximum(bound, np.finfo(np.float64).tiny)))
        assert ratio <= 2.0, (q, ks[q], ratio)
    if inplace:
        assert np.array_equal(out[:, offs[-2]:], G[:, offs[-2]:])


def test_two_level_wide_pivots_all_digit():
    """Two-level solves whose pivots span several tiles, all contractions as
    digit products: complex b = 32 (64-column pivots, 2 tiles per side, inner
    solve in shared memory) in the full-block and block-oriented forms,
    complex b = 48 (96-column pivots, 3 tiles) and real b = 64 (128-column
    pivots, 2 tiles) in the full-block form (inner solve in global memory);
    eigenvalues against the construction and the oracle."""
    jj = require_gpu()
    P = synth.make_workload("plain_c128_n128", n=288)
    ref = oracle.solve_plain(P.G, P.J)
    tol = eig_rel_tol(P.G)
    for bw, strategy in ((32, jj.JJ_FULL_BLOCK), (32, jj.JJ_BLOCK_ORIENTED), (48, jj.JJ_FULL_BLOCK)):
        got = solve_gpu(P.G, P.J, block_width=bw, gemm=1, block_strategy=strategy)
        assert got["info"]["status"] == 0, (bw, strategy)
        assert max_rel_err(got["lam"], ref["lam"]) <= tol, (bw, strategy)
        assert max_rel_err(got["lam"], P.lam_exact) <= tol, (bw, strategy)
    Q = synth.make_workload("blocked_f64_n2048_b32", n=512)
    got = solve_gpu(Q.G, Q.J, block_width=64, gemm=1)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], Q.lam_exact) <= eig_rel_tol(Q.G)


def test_graded_complex_b64_three_level_all_digit():
    """The graded complex recipe at its block width b = 64 (128-column outer
    pivots, 4 tiles per side, through the three-level form with inner blocks
    of 16), all contractions as digit products: eigenvalues within the graded
    tolerance of the oracle's."""
    require_gpu()
    P = synth.make_workload("graded_c128_n4096_b64", n=512)
    ref = oracle.solve_plain(P.G, P.J)
    got = solve_gpu(P.G, P.J, block_width=64, inner_block_width=16, gemm=1)
    assert got["info"]["status"] == 0
    assert max_rel_err(got["lam"], ref["lam"]) <= 1e-10
