"""Seeded synthetic inputs for the one-sided hyperbolic (J-)Jacobi eigensolver.

This module serves both the CUDA path (tests, bench) and the CPU oracle. It
holds only the *construction* of inputs, never the solver's arithmetic: the
random plane rotations it applies have angles drawn from a random generator,
not computed from the data.

Construction (the paper tests on random eigenvalues in a range, transformed by
random reflectors, Sec. 3.5; these recipes stand in for those LAPACK testing
matrices):

  1. Q is Haar-unitary (orthogonal in the real case): QR of a Ginibre matrix
     with the phases of diag(R) divided out.
  2. |Lambda| is log-uniform in [lo, hi]; the signs of Lambda are J.
  3. J is sorted as diag(+I_nu, -I_{n-nu}) (the ordering of Sec. 2.3).
  4. W is a product of random J-unitary plane rotations: a uniform random pair
     (r != s); trigonometric (2.1)/(2.2) when J_rr = J_ss, with angle
     phi ~ U[0, 2 pi) and phase alpha ~ U[0, 2 pi); hyperbolic (2.7) otherwise,
     with sinh ~ U[-smax, smax] and a random phase.
  5. G = Q |Lambda|^{1/2} W, so that H = G J G^* = Q (J |Lambda|) Q^*: the
     exact eigenvalues are J_ii |Lambda_ii| (W J W^* = J because W is
     J-unitary).
  6. Optionally G <- D1 G D2 with D1, D2 diagonal, log-uniform (graded case);
     the eigenvalues are then no longer known by construction.

Precision: 'ld' builds G0 = Q|Lambda|^{1/2} and applies W in numpy long double
(80-bit on x86-64, binary128 on aarch64) before rounding G to float64; 'f64'
does everything in float64 (used for the large workloads, where the
construction pin is not needed).

Storage: G is returned as a Fortran-ordered (column-major) numpy array of
complex128 or float64, shape (m, n), with m = n.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

__all__ = [
    "Problem",
    "WORKLOADS",
    "make_problem",
    "make_workload",
    "make_batched",
    "haar_unitary",
    "random_rotation_draws",
]


@dataclasses.dataclass
class Problem:
    """One synthetic input: G (m x n, column-major), J (int8 +-1), metadata."""

    G: np.ndarray
    J: np.ndarray
    lam_exact: Optional[np.ndarray]  # J_ii |Lambda_ii| when known by construction
    name: str
    seed: int
    graded: bool = False

    @property
    def n(self) -> int:
        return self.G.shape[1]

    @property
    def m(self) -> int:
        return self.G.shape[0]

    @property
    def is_complex(self) -> bool:
        return np.iscomplexobj(self.G)


# The five workloads. Sizes, ranges and rotation counts are those of the
# published configurations; block widths are the solver settings they name.
WORKLOADS = {
    # plain non-blocked, complex128, n = 128, J = (+80, -48)
    "plain_c128_n128": dict(n=128, cplx=True, npos=80, lam=(1e-3, 1e3),
                            rots=256, smax=2.0, seed=1000, block=0),
    # blocked two-level, float64, n = 2048, b = 32
    "blocked_f64_n2048_b32": dict(n=2048, cplx=False, npos=1024, lam=(1e-4, 1e4),
                                  rots=4096, smax=3.0, seed=1001, block=32),
    # blocked, complex128, n = 4096, b = 64, graded D1 B D2
    "graded_c128_n4096_b64": dict(n=4096, cplx=True, npos=2560, lam=(1e-3, 1e3),
                                  rots=256, smax=2.0, seed=1002, block=64,
                                  grade=(1e-5, 1e5)),
    # batched: 512 complex128 problems, n ~ U[32, 512]
    "batched_c128_512x": dict(count=512, nrange=(32, 512), cplx=True,
                              posfrac=(0.2, 0.8), lam=(1e-3, 1e3), rots=256,
                              smax=2.0, seed=1003),
    # three-level, float64, n = 16384, b = 128, inner 16-column blocks
    "threelevel_f64_n16384_b128": dict(n=16384, cplx=False, npos=8192,
                                       lam=(1e-6, 1e6), rots=65536, smax=2.0,
                                       seed=1004, block=128, inner=16),
}


def haar_unitary(n: int, rng: np.random.Generator, cplx: bool) -> np.ndarray:
    """Haar-distributed unitary (orthogonal) matrix via QR of a Ginibre matrix."""
    if cplx:
        Z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2.0)
    else:
        Z = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    ph = d / np.abs(d)
    return Q * ph[None, :]


def random_rotation_draws(n: int, J: np.ndarray, count: int, smax: float,
                          rng: np.random.Generator, cplx: bool):
    """Draw `count` random plane rotations: (r, s, hyperbolic?, angle-or-sinh, phase)."""
    out = []
    if n < 2:
        return out
    for _ in range(count):
        r = int(rng.integers(0, n))
        s = int(rng.integers(0, n - 1))
        if s >= r:
            s += 1
        hyper = bool(J[r] != J[s])
        if hyper:
            par = float(rng.uniform(-smax, smax))
        else:
            par = float(rng.uniform(0.0, 2.0 * math.pi))
        ph = float(rng.uniform(0.0, 2.0 * math.pi)) if cplx else 0.0
        out.append((r, s, hyper, par, ph))
    return out


def _apply_draws(G: np.ndarray, draws, cplx: bool) -> None:
    """G <- G * W_1 * W_2 ... with each W_k a random J-unitary rotation (in place).

    Trigonometric form (2.2): columns (g_r, g_s) <- (c g_r - e^{-ia} s g_s,
    e^{ia} s g_r + c g_s); hyperbolic form (2.7) with a phase:
    (g_r, g_s) <- (ch g_r + e^{-ia} sh g_s, e^{ia} sh g_r + ch g_s).
    """
    ld = G.dtype in (np.longdouble, np.clongdouble)
    one = np.longdouble(1) if ld else 1.0
    for (r, s, hyper, par, ph) in draws:
        if hyper:
            sh = one * par
            ch = np.sqrt(one + sh * sh)
            a, b = ch, sh
        else:
            phi = one * par
            a, b = np.cos(phi), np.sin(phi)
        gr = G[:, r].copy()
        gs = G[:, s].copy()
        if cplx:
            e = np.exp(1j * (one * ph)) if not ld else (np.cos(one * ph) + 1j * np.sin(one * ph))
            ec = np.conj(e)
        else:
            e = ec = one
        if hyper:
            G[:, r] = a * gr + ec * b * gs
            G[:, s] = e * b * gr + a * gs
        else:
            G[:, r] = a * gr - ec * b * gs
            G[:, s] = e * b * gr + a * gs


def _log_uniform(rng: np.random.Generator, lo: float, hi: float, size: int) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def make_problem(n: int, cplx: bool, npos: int, lam: Tuple[float, float], rots: int,
                 smax: float, seed, grade: Optional[Tuple[float, float]] = None,
                 precision: str = "ld", name: str = "", m: Optional[int] = None) -> Problem:
    """Build one problem by the recipe in the module docstring.

    `seed` may be an int or a tuple (fed to numpy's SeedSequence / PCG64).
    m >= n gives a tall G (m rows): Q is then m x m and G0 = Q[:, :n] |Lambda|^{1/2}.
    """
    m = n if m is None else m
    assert m >= n >= 1 and 0 <= npos <= n
    rng = np.random.Generator(np.random.PCG64(seed))
    Q = haar_unitary(m, rng, cplx)[:, :n]
    mag = _log_uniform(rng, lam[0], lam[1], n)
    J = np.ones(n, dtype=np.int8)
    J[npos:] = -1
    draws = random_rotation_draws(n, J, rots, smax, rng, cplx)
    if precision == "ld":
        dt = np.clongdouble if cplx else np.longdouble
        G = Q.astype(dt) * np.sqrt(mag.astype(np.longdouble))[None, :]
    else:
        G = Q * np.sqrt(mag)[None, :]
    _apply_draws(G, draws, cplx)
    G = np.asfortranarray(G.astype(np.complex128 if cplx else np.float64))
    lam_exact = J.astype(np.float64) * mag
    graded = grade is not None
    if graded:
        d1 = _log_uniform(rng, grade[0], grade[1], m)
        d2 = _log_uniform(rng, grade[0], grade[1], n)
        G = np.asfortranarray(d1[:, None] * G * d2[None, :])
        lam_exact = None
    return Problem(G=G, J=J, lam_exact=lam_exact, name=name or f"n{n}", seed=seed,
                   graded=graded)


def make_workload(name: str, n: Optional[int] = None, precision: Optional[str] = None,
                  rots: Optional[int] = None) -> Problem:
    """One of the single-problem workloads, optionally scaled down to order n.

    Scaling keeps the J split fraction, the eigenvalue range, the grading and
    the rotations-per-column ratio of the full-size recipe.
    """
    w = WORKLOADS[name]
    assert "count" not in w, "use make_batched for the batched workload"
    N = w["n"]
    nn = N if n is None else n
    npos = int(round(w["npos"] * nn / N))
    nrots = w["rots"] if n is None else max(1, int(round(w["rots"] * nn / N)))
    if rots is not None:
        nrots = rots
    prec = precision or ("ld" if nn <= 1024 else "f64")
    return make_problem(nn, w["cplx"], npos, w["lam"], nrots, w["smax"], w["seed"],
                        grade=w.get("grade"), precision=prec,
                        name=f"{name}@n{nn}")


def make_batched(count: Optional[int] = None, nrange: Optional[Tuple[int, int]] = None,
                 precision: str = "f64") -> List[Problem]:
    """The batched workload: `count` independent complex problems of uneven order.

    Problem i uses seed (1003, i). Orders n ~ U[nrange] and the +1 fraction of J
    ~ U[0.2, 0.8] are drawn from seed 1003 itself.
    """
    w = WORKLOADS["batched_c128_512x"]
    cnt = w["count"] if count is None else count
    lo, hi = w["nrange"] if nrange is None else nrange
    rng = np.random.Generator(np.random.PCG64(w["seed"]))
    ns = rng.integers(lo, hi + 1, size=w["count"])[:cnt]
    fr = rng.uniform(w["posfrac"][0], w["posfrac"][1], size=w["count"])[:cnt]
    out = []
    for i in range(cnt):
        n = int(ns[i])
        npos = int(round(fr[i] * n))
        out.append(make_problem(n, True, npos, w["lam"], w["rots"], w["smax"],
                                (w["seed"], i), precision=precision,
                                name=f"batched[{i}]@n{n}"))
    return out
