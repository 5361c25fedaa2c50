"""How many 7-bit digits per operand the digit-product block update needs to be
as accurate as FP64 on the graded inputs: the evidence behind keeping the
update in FP64 in the accurate (hybrid) form.

This is a study, not a parity test: it models the digit scheme of the update
in exact integer arithmetic and compares it, entry by entry, with FP64's own
error bound for the same update on a real iterate of the method.

The scheme modelled (the update [G_i G_j] <- [G_i G_j] W_P of (2.9), written
as X + X D with D = W_P - I on the real form X = [Re G_P, Im G_P]):
  * X is scaled by a power of two per column (its largest exponent), then
    each row of the scaled X gets its own exponent r_l;
  * D is multiplied by the same column powers (rows of D), and each column of
    the result gets its own exponent w_j;
  * both are cut into s truncated 7-bit digits relative to those exponents,
    and the digit products with t + u <= s + 1 are summed exactly.
Its error is relative to 2^(r_l + w_j), a row scale times a column scale,
while FP64's bound is u (|x_lj| + sum_a |x_la| |d_aj|) per entry. On graded
iterates the two differ by orders of magnitude for many entries.

The iterate: the oracle's two-level full-block reference on the graded complex
recipe at n = 128, b = 8, after 75 parallel steps (5 sweeps); its first pivot
pair of the next step (48 rows kept, so that the exact arithmetic stays
quick)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def _exps(a):
    """Smallest e with |a| < 2^e, per entry (-1021 for zeros)."""
    m = np.abs(a)
    e = np.frexp(m)[1].astype(np.int64)
    e[m == 0] = -1021
    return e


def _fixed(v: float, e: int, bits: int) -> int:
    """Signed floor(|v| 2^(bits - e)) for |v| < 2^e, exactly."""
    fr = Fraction(v) * Fraction(2) ** (bits - e)
    q = abs(fr.numerator) // fr.denominator
    return q if v >= 0 else -q


def _digit_update(X, D, s):
    """X D with s digits per operand, as exact Fractions."""
    F = 7 * s
    ce = _exps(X).max(axis=0)
    Xh = np.ldexp(X, -ce[None, :])
    r = _exps(Xh).max(axis=1)
    Dp = np.ldexp(D, ce[:, None])
    w = _exps(Dp).max(axis=0)
    qx = [[_fixed(float(Xh[l, a]), int(r[l]), F) for a in range(X.shape[1])] for l in range(X.shape[0])]
    qd = [[_fixed(float(Dp[a, j]), int(w[j]), F) for j in range(D.shape[1])] for a in range(D.shape[0])]

    def digit(q, t):
        d = (abs(q) >> (F - 7 * t)) & 127
        return d if q >= 0 else -d

    dx = [np.array([[digit(q, t) for q in row] for row in qx], dtype=object) for t in range(1, s + 1)]
    dd = [np.array([[digit(q, t) for q in row] for row in qd], dtype=object) for t in range(1, s + 1)]
    acc = np.zeros((X.shape[0], D.shape[1]), dtype=object)
    for t in range(1, s + 1):
        for u in range(1, s + 2 - t):
            acc = acc + dx[t - 1].dot(dd[u - 1]) * (1 << (7 * (2 * s - t - u)))
    out = np.empty(acc.shape, dtype=object)
    for (l, j), v in np.ndenumerate(acc):
        out[l, j] = Fraction(int(v)) * Fraction(2) ** (int(r[l]) + int(w[j]) - 14 * s)
    return out


@pytest.fixture(scope="module")
def graded_pivot():
    P = synth.make_workload("graded_c128_n4096_b64", n=128)
    st = oracle.solve_blocked(P.G, P.J, 8, max_steps=75)
    G, nbl, sizes = st["Gt"], st["nbl"], st["sizes"]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    i, j = 0, nbl // 2
    cols = np.r_[offs[i]:offs[i + 1], offs[j]:offs[j + 1]]
    GP = G[:, cols]
    R = oracle.cholesky_upper(oracle.gram(GP))
    W = oracle.inner_solve(R, P.J[cols])["W"]
    X = np.concatenate([GP.real, GP.imag], axis=1)[:48]
    W2 = np.block([[W.real, W.imag], [-W.imag, W.real]])
    D = W2 - np.eye(W2.shape[0])
    Xf = [[Fraction(float(v)) for v in row] for row in X]
    Df = [[Fraction(float(v)) for v in row] for row in D]
    exact = np.empty((X.shape[0], D.shape[1]), dtype=object)
    for l in range(X.shape[0]):
        for c in range(D.shape[1]):
            exact[l, c] = sum(Xf[l][a] * Df[a][c] for a in range(D.shape[0]))
    # FP64's own error scale for X + X D, entry by entry
    bound = (np.abs(X) @ np.abs(D)) * 2.0 ** -53 + np.abs(X) * 2.0 ** -53
    return X, D, exact, bound


def _ratio(graded_pivot, s):
    X, D, exact, bound = graded_pivot
    C = _digit_update(X, D, s)
    err = np.array([[float(abs(C[l, c] - exact[l, c])) for c in range(D.shape[1])]
                    for l in range(X.shape[0])])
    return err / bound


def test_eight_digits_miss_fp64_accuracy_on_graded_iterates(graded_pivot):
    """The 8-digit update of the all-digit form exceeds FP64's per-entry bound
    on a large share of the entries: why it misses the graded tolerance."""
    ratio = _ratio(graded_pivot, 8)
    assert np.mean(ratio > 1) > 0.05 and np.max(ratio) > 100


def test_twelve_digits_meet_fp64_accuracy_on_graded_iterates(graded_pivot):
    """With 12 digits per operand (84 bits) every entry is within FP64's
    bound: the digit count an accurate all-digit update would need."""
    ratio = _ratio(graded_pivot, 12)
    assert np.max(ratio) <= 1.0
