"""Batched solve (many independent problems of uneven order per launch) against
the oracle, against eigenvalues known by construction, and against the single
solve of each problem (the batched plan runs the same per-pair arithmetic, so
the results agree bit for bit)."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import eig_rel_tol, max_rel_err
from tests.gpu_util import from_dev, require_gpu, solve_gpu, to_dev

pytestmark = pytest.mark.gpu


def _problems(cplx, ns, seed):
    out = []
    for i, n in enumerate(ns):
        npos = max(0, min(n, int(round(n * (0.2 + 0.6 * ((i * 7919) % 97) / 96)))))
        out.append(synth.make_problem(n, cplx, npos, (1e-3, 1e3), 2 * n, 2.0, seed=(seed, i),
                                      precision="f64"))
    return out


def _run(jj, probs, cplx, gemm, block_width=0, max_sweeps=0):
    import torch

    mmax = max(P.m for P in probs)
    nmax = max(P.n for P in probs)
    Gs = [to_dev(P.G) for P in probs]
    lam = torch.full((sum(P.n for P in probs),), float("nan"), dtype=torch.float64, device="cuda")
    with jj.Handle(mmax, nmax, jj.JJ_C128 if cplx else jj.JJ_F64, block_width=block_width,
                   gemm=gemm, max_sweeps=max_sweeps) as h:
        rc, infos = h.jjacobi_solve_batched(Gs, [P.J for P in probs], lam, allow=(0, 2))
    torch.cuda.synchronize()
    lam = lam.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([P.n for P in probs])])
    return rc, infos, [lam[offs[i]:offs[i + 1]] for i in range(len(probs))], [from_dev(G) for G in Gs]


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("gemm", [0, 1, 2])
def test_batched_uneven_matches_oracle(cplx, gemm):
    jj = require_gpu()
    ns = [1, 2, 3, 5, 17, 33, 40, 64, 71, 96, 8, 129]
    probs = _problems(cplx, ns, 4242 + cplx)
    rc, infos, lams, Gts = _run(jj, probs, cplx, gemm)
    assert rc == 0, jj.status_string(rc)
    for P, lam, info, Gt in zip(probs, lams, infos, Gts):
        d = info.as_dict()
        assert d["status"] == 0
        assert np.all(np.isfinite(lam))
        assert np.all(np.sign(lam) == P.J)  # caller column order, signs by J
        tol = eig_rel_tol(P.G)
        ref = oracle.solve_plain(P.G, P.J)
        assert max_rel_err(lam, ref["lam"]) <= tol
        assert max_rel_err(np.sort(lam), np.sort(P.lam_exact)) <= tol
        # lambda is J ||g~||^2 of the returned G~
        nrm = np.sum(np.abs(Gt) ** 2, axis=0) * P.J
        assert np.max(np.abs(nrm - lam) / np.abs(lam)) <= 1e-13


@pytest.mark.parametrize("gemm", [0, 1, 2])
def test_batched_equals_single_solves(gemm):
    """Per problem, the batched plan is the single plan (same partition, same
    ordering, deterministic kernels): G~ agrees exactly."""
    jj = require_gpu()
    cplx = True
    ns = [24, 48, 70, 33]
    probs = _problems(cplx, ns, 777)
    b = 16
    rc, infos, lams, Gts = _run(jj, probs, cplx, gemm, block_width=b)
    assert rc == 0
    _, _, _, again = _run(jj, probs, cplx, gemm, block_width=b)
    assert all(np.array_equal(x, y) for x, y in zip(Gts, again))  # deterministic
    for P, lam, Gt, info in zip(probs, lams, Gts, infos):
        single = solve_gpu(P.G, P.J, block_width=b, gemm=gemm)
        assert single["info"]["sweeps"] == info.as_dict()["sweeps"]
        assert np.array_equal(single["Gt"], Gt)
        assert np.array_equal(single["lam"], lam)


def test_batched_plan_reuse_and_shape_change():
    """A second call with the same shapes reuses the plan (and its graph); a
    call with other shapes rebuilds it; a single solve on the same handle still works."""
    jj = require_gpu()
    import torch

    probs = _problems(True, [20, 31, 12], 91)
    probs2 = _problems(True, [40, 9], 92)
    with jj.Handle(64, 64, jj.JJ_C128, gemm=1) as h:
        for batch in (probs, probs, probs2):
            Gs = [to_dev(P.G) for P in batch]
            lam = np.zeros(sum(P.n for P in batch))
            rc, infos = h.jjacobi_solve_batched(Gs, [P.J for P in batch], lam)
            assert rc == 0
            off = 0
            for P in batch:
                assert max_rel_err(np.sort(lam[off:off + P.n]), np.sort(P.lam_exact)) <= eig_rel_tol(P.G)
                off += P.n
        P = _problems(True, [64], 93)[0]  # the handle's own single-solve shape
        Gd = to_dev(P.G)
        h.jjacobi_solve(Gd, Gd.stride(1), P.J)
        lam = torch.empty(P.n, dtype=torch.float64, device="cuda")
        h.jjacobi_extract(lam)
        assert max_rel_err(np.sort(lam.cpu().numpy()), np.sort(P.lam_exact)) <= eig_rel_tol(P.G)


def test_batched_rejects_bad_arguments():
    jj = require_gpu()
    probs = _problems(False, [10, 20], 5)
    with jj.Handle(16, 16, jj.JJ_F64) as h:  # second problem larger than the handle allows
        Gs = [to_dev(P.G) for P in probs]
        with pytest.raises(jj.JJError):
            h.jjacobi_solve_batched(Gs, [P.J for P in probs])
    with jj.Handle(32, 32, jj.JJ_F64) as h:
        Gs = [to_dev(P.G) for P in probs]
        bad = [P.J.copy() for P in probs]
        bad[1][3] = 0
        with pytest.raises(jj.JJError):
            h.jjacobi_solve_batched(Gs, bad)


def test_batched_workload_sample():
    """The 512-problem workload's generator, first 24 problems (orders drawn
    from U[32, 512]): eigenvalues by construction, plus the oracle on the
    smallest three."""
    jj = require_gpu()
    probs = synth.make_batched(count=24)
    rc, infos, lams, _ = _run(jj, probs, True, 1)
    assert rc == 0
    for P, lam in zip(probs, lams):
        assert max_rel_err(np.sort(lam), np.sort(P.lam_exact)) <= eig_rel_tol(P.G)
    for i in np.argsort([P.n for P in probs])[:3]:
        ref = oracle.solve_plain(probs[i].G, probs[i].J)
        assert max_rel_err(lams[i], ref["lam"]) <= eig_rel_tol(probs[i].G)


def test_batched_ill_conditioned_problem_finished_by_plain_method():
    """Problem 30 of the 512-problem workload (n = 32, scaled condition ~6e9):
    its single pivot is the whole problem, whose Gram block is not positive
    definite in FP64; the batch finishes it with the plain method (block_width
    0 in its info) and its eigenvalues match the plain oracle."""
    jj = require_gpu()
    allp = synth.make_batched(count=31)
    probs = [allp[0], allp[30], allp[5]]
    rc, infos, lams, _ = _run(jj, probs, True, 1)
    assert rc == 0
    d = infos[1].as_dict()
    assert d["status"] == 0 and d["block_width"] == 0
    assert infos[0].as_dict()["block_width"] > 0
    for P, lam in zip(probs, lams):
        ref = oracle.solve_plain(P.G, P.J)
        assert max_rel_err(lam, ref["lam"]) <= eig_rel_tol(P.G)


def test_batched_autotuned_widths_per_size_class():
    """block_width = JJ_BLOCK_AUTO: one width per size class (floor(log2 n)),
    chosen by timing one sweep of that class's sub-batch per candidate; results
    as accurate as with fixed widths, and the second call reuses the choice."""
    jj = require_gpu()
    import torch

    probs = _problems(True, [20, 28, 40, 60, 100, 120, 130, 200], 314)
    mmax, nmax = max(P.m for P in probs), max(P.n for P in probs)
    with jj.Handle(mmax, nmax, jj.JJ_C128, block_width=jj.JJ_BLOCK_AUTO, gemm=1) as h:
        for call in range(2):
            Gs = [to_dev(P.G) for P in probs]
            lam = torch.empty(sum(P.n for P in probs), dtype=torch.float64, device="cuda")
            rc, infos = h.jjacobi_solve_batched(Gs, [P.J for P in probs], lam)
            assert rc == 0
            widths = [i.as_dict()["block_width"] for i in infos]
            if call == 0:
                first = widths
            assert widths == first
            lam = lam.cpu().numpy()
            off = 0
            for P, w in zip(probs, widths):
                assert w in (0, 8, 16) or w == (P.n + 1) // 2
                assert max_rel_err(np.sort(lam[off:off + P.n]), np.sort(P.lam_exact)) <= eig_rel_tol(P.G)
                off += P.n
