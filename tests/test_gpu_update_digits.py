"""The split-precision block update (2.9) on the tensor cores, through the C ABI:
entry-by-entry accuracy against FP64's own error bound on a graded iterate of
the method, the digit counts, in-place and out-of-place forms, ragged tiles
and more work items than the GPU has multiprocessors."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import U64, eig_rel_tol, max_rel_err
from tests.gpu_util import from_dev, require_gpu, solve_gpu, to_dev

pytestmark = pytest.mark.gpu


def _pivot(G, pd):
    a, na, b, nb = pd
    return np.concatenate([G[:, a:a + na], G[:, b:b + nb]], axis=1)


def _real_form(X, W):
    """[Xr Xi] and [[Wr, Wi], [-Wi, Wr]] in long double: Y = X W as real blocks."""
    L = np.longdouble
    Xr = np.concatenate([X.real, X.imag], axis=1).astype(L)
    W2 = np.block([[W.real, W.imag], [-W.imag, W.real]]).astype(L)
    return Xr, W2


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
    dt = jj.JJ_C128 if np.iscomplexobj(G) else jj.JJ_F64
    jj.jjk_update(dt, jj.JJ_GEMM_OZAKI_FP16, Gs, Gd, Gs.stride(1), G.shape[0], pd, len(pairs),
                  Wd, kmax)
    torch.cuda.synchronize()
    return from_dev(Gd)


@pytest.mark.parametrize("b", [8, 16])
def test_update_within_fp64_entry_bound_on_graded_iterate(b):
    """On a real iterate of the method on the graded complex recipe (the
    oracle's blocked reference after 75 parallel steps, n = 192, so 2 row
    tiles with a ragged one), every entry of [G_i G_j] W_P computed from 11
    balanced 8-bit digits per operand is within twice FP64's own bound
    u (|x_lj| + sum_a |x_la| |w_aj - delta_aj|) of the exact product (long
    double): the correction form's error u sum |x||d| plus the final
    rounding. With one exponent per row and column a 56-bit update misses
    this bound by up to 1e6 (tests/test_digit_update_accuracy_study.py)."""
    jj = require_gpu()
    P = synth.make_workload("graded_c128_n4096_b64", n=192)
    st = oracle.solve_blocked(P.G, P.J, b, max_steps=75)
    G, nbl, sizes = st["Gt"], st["nbl"], st["sizes"]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    tab = jj.jjacobi_schedule(nbl, 0, 1)
    pairs = [[offs[i], sizes[i], offs[j], sizes[j]] for i, j in tab[0]]
    kmax = 2 * int(max(sizes))
    Ws = []
    for p in pairs:
        cols = np.r_[p[0]:p[0] + p[1], p[2]:p[2] + p[3]]
        R = oracle.cholesky_upper(oracle.gram(G[:, cols]))
        Ws.append(oracle.inner_solve(R, P.J[cols])["W"])
    for inplace in (False, True):
        out = _update(jj, G, pairs, Ws, kmax, inplace)
        worst = 0.0
        for q, p in enumerate(pairs):
            X = _pivot(G, p)
            Xr, W2 = _real_form(X, Ws[q])
            exact = Xr @ W2
            D = np.abs(W2 - np.eye(W2.shape[0], dtype=W2.dtype))
            bound = (np.abs(Xr) @ D + np.abs(Xr)) * U64
            Y = _pivot(out, p)
            got = np.concatenate([Y.real, Y.imag], axis=1).astype(np.longdouble)
            ratio = np.abs(got - exact) / np.maximum(bound, np.finfo(np.float64).tiny)
            worst = max(worst, float(np.max(ratio)))
        assert worst <= 2.0, (inplace, worst)


def test_update_many_items_ragged_real_in_place():
    """Real pivots of up to 64 columns, 3 row tiles with a ragged last one, and
    200 pairs (more work items than multiprocessors, so every persistent block
    takes several pairs): in place, every entry within twice FP64's own bound
    of the exact product (long double)."""
    jj = require_gpu()
    rng = np.random.default_rng(41)
    m, nblk = 300, 400
    sizes = rng.integers(20, 33, size=nblk)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    n = int(offs[-1])
    G = np.asfortranarray(rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-3, 3, size=(m, 1)))
    perm = rng.permutation(nblk)
    pairs = [[offs[perm[2 * q]], sizes[perm[2 * q]], offs[perm[2 * q + 1]], sizes[perm[2 * q + 1]]]
             for q in range(nblk // 2)]
    kmax = 64
    Ws = []
    for p in pairs:
        k = p[1] + p[3]
        Ws.append(np.eye(k) + 1e-2 * rng.standard_normal((k, k)) * 10.0 ** rng.uniform(-2, 2, size=(1, k)))
    out = _update(jj, G, pairs, Ws, kmax, True)
    L = np.longdouble
    for q in list(range(0, len(pairs), 9)) + [len(pairs) - 1]:  # a sample (long double is slow)
        p = pairs[q]
        X = _pivot(G, p)
        exact = X.astype(L) @ Ws[q].astype(L)  # the product of the FP64 operands
        bound = (np.abs(X) @ np.abs(Ws[q] - np.eye(Ws[q].shape[0])) + np.abs(X)) * U64
        err = np.abs(_pivot(out, p).astype(L) - exact)
        assert np.max(err / bound) <= 2.0, q
    # columns outside every pair are untouched
    used = np.zeros(n, dtype=bool)
    for p in pairs:
        used[p[0]:p[0] + p[1]] = True
        used[p[2]:p[2] + p[3]] = True
    assert np.array_equal(out[:, ~used], G[:, ~used])


def test_digit_counts():
    """Every digit count of the update runs (one phase of TMEM groups up to 6
    digits, two phases above): the eigenvalue error falls as digits are added,
    and with 11 the all-digit solve meets the scaled-condition bound."""
    require_gpu()
    P = synth.make_workload("plain_c128_n128", n=96)
    errs = {}
    for digits in (3, 4, 6, 7, 9, 11):
        got = solve_gpu(P.G, P.J, block_width=16, gemm=1, ozaki_slices=digits, max_sweeps=40,
                        allow=(0, 2))
        errs[digits] = max_rel_err(got["lam"], P.lam_exact)
        assert np.isfinite(errs[digits])
        if digits == 11:
            assert got["info"]["status"] == 0
    print("relative eigenvalue error by digits:", errs)
    assert errs[11] <= eig_rel_tol(P.G)
    assert errs[3] > errs[4] > errs[11] or errs[4] <= eig_rel_tol(P.G)
    assert errs[6] >= errs[9] or errs[9] <= eig_rel_tol(P.G)


def test_rejects_more_than_eleven_digits():
    jj = require_gpu()
    with pytest.raises(jj.JJError):
        jj.Handle(128, 128, jj.JJ_C128, block_width=16, gemm=1, ozaki_slices=12)
