"""Parity at the published full sizes, in the launch configurations bench.py
times, through properties that hold at any size (the oracle's full solve of
these inputs takes hours):

- the solve is a J-unitary transformation: G~ J G~^* = G J G^* (checked on
  sampled vectors on the host, relative to the rounding scale of both sides);
- the columns of G~ are orthogonal (sampled pairs, the convergence criterion);
- lambda_i = J_ii ||g~_i||^2 carries the sign of J_ii;
- eigenvalues known by construction where the recipe gives them, and agreement
  with the independent plain (non-blocked) kernel path on the graded input.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._util import eig_rel_tol, max_rel_err
from tests.gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _solve(jj, P, **kw):
    import torch

    Gd = to_dev(P.G)
    m, n = P.G.shape
    with jj.Handle(m, n, jj.JJ_C128 if P.is_complex else jj.JJ_F64, **kw) as h:
        info = h.jjacobi_solve(Gd, Gd.stride(1), P.J).as_dict()
        lam = torch.empty(n, dtype=torch.float64, device="cuda")
        h.jjacobi_extract(lam)
    return info, lam.cpu().numpy(), from_dev(Gd)


def _check_properties(P, Gt, lam, seed, nvec=4, npairs=400):
    rng = np.random.default_rng(seed)
    G = np.asarray(P.G)
    J = np.asarray(P.J, dtype=np.float64)
    # J-unitary invariance on sampled vectors: G~ J G~^* x = G J G^* x
    for _ in range(nvec):
        x = rng.standard_normal(G.shape[0]) + (1j * rng.standard_normal(G.shape[0]) if P.is_complex else 0)
        a = G @ (J * (G.conj().T @ x))
        b = Gt @ (J * (Gt.conj().T @ x))
        # rounding scale of both sides: |G| |G|^T |x| + |G~| |G~|^T |x|
        scale = np.abs(G) @ (np.abs(G).T @ np.abs(x)) + np.abs(Gt) @ (np.abs(Gt).T @ np.abs(x))
        assert np.max(np.abs(a - b) / scale) <= 1e-10
    # orthogonality of sampled column pairs
    nrm = np.linalg.norm(Gt, axis=0)
    i = rng.integers(0, G.shape[1], size=npairs)
    j = rng.integers(0, G.shape[1], size=npairs)
    keep = i != j
    i, j = i[keep], j[keep]
    cos = np.abs(np.sum(Gt[:, i].conj() * Gt[:, j], axis=0)) / (nrm[i] * nrm[j])
    assert np.max(cos) <= 8 * oracle.TOL_DEFAULT
    # lambda = J ||g~||^2, signs by J
    assert np.all(np.sign(lam) == P.J)
    assert np.max(np.abs(lam - J * nrm ** 2) / np.abs(lam)) <= 1e-13


def test_headline_graded_complex_n4096_bench_configuration():
    """The graded complex workload at n = 4096 as bench.py runs it (b = 16,
    block-oriented, digit Gram + FP64 update), against the plain kernel path."""
    jj = require_gpu()
    P = synth.make_workload("graded_c128_n4096_b64", precision="f64")
    info, lam, Gt = _solve(jj, P, block_width=16, gemm=jj.JJ_GEMM_OZAKI_GRAM,
                           block_strategy=jj.JJ_BLOCK_ORIENTED)
    assert info["status"] == 0
    _check_properties(P, Gt, lam, seed=1)
    pinfo, plam, _ = _solve(jj, P, block_width=0)
    assert pinfo["status"] == 0
    assert max_rel_err(lam, plam) <= 1e-10


def test_blocked_real_n2048_b32_full_size():
    """The real two-level workload at n = 2048, b = 32 (64 blocks, 63 steps):
    eigenvalues by construction (to the scaled-condition bound) and the
    properties above."""
    jj = require_gpu()
    P = synth.make_workload("blocked_f64_n2048_b32", precision="f64")
    info, lam, Gt = _solve(jj, P, block_width=32, gemm=jj.JJ_GEMM_FP64)
    assert info["status"] == 0 and info["nbl"] == 64
    _check_properties(P, Gt, lam, seed=2)
    assert max_rel_err(lam, P.lam_exact) <= eig_rel_tol(P.G)


def test_batched_512_problems_full_size():
    """All 512 problems of the batched workload in one call, as bench.py runs
    it (digit forms): every problem converged (the ill-conditioned ones via the
    plain method), eigenvalues by construction to each problem's bound."""
    jj = require_gpu()
    import torch

    probs = synth.make_batched(precision="f64")
    Gs = [to_dev(P.G) for P in probs]
    lam = torch.empty(sum(P.n for P in probs), dtype=torch.float64, device="cuda")
    with jj.Handle(max(P.m for P in probs), max(P.n for P in probs), jj.JJ_C128,
                   gemm=jj.JJ_GEMM_OZAKI_FP16) as h:
        rc, infos = h.jjacobi_solve_batched(Gs, [P.J for P in probs], lam)
    assert rc == 0
    lam = lam.cpu().numpy()
    off = 0
    for P, inf in zip(probs, infos):
        assert inf.status == 0
        lp = lam[off:off + P.n]
        off += P.n
        assert np.all(np.sign(lp) == P.J)
        assert max_rel_err(lp, P.lam_exact) <= eig_rel_tol(P.G)
