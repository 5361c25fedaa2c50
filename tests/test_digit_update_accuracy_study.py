"""How many digits per operand the digit-product block update needs to be as
accurate as FP64 on the graded inputs: the evidence behind the update's digit
count.

This is a study, not a parity test: it models the digit scheme of the update
in exact integer arithmetic and compares it, entry by entry, with FP64's own
error bound for the same update on a real iterate of the method.

The scheme modelled (the update [G_i G_j] <- [G_i G_j] W_P of (2.9), written
as X + X D with D = W_P - I on the real form X = [Re G_P, Im G_P]):
  * X is scaled by a power of two per column (its largest exponent), then
    each row of the scaled X gets its own exponent r_l;
  * D is multiplied by the same column powers (rows of D), and each column of
    the result gets its own exponent w_j;
  * both are cut into s balanced 8-bit digits relative to those exponents
    (the truncated image V = +-floor(|v| 2^(86 - e)) written as
    sum (u_i - 128) 256^i with the bytes u_i of V + sum 128 * 256^i), and the
    digit products with t + u <= s + 1 are summed exactly.
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


def _fixed(v: float, e: int) -> int:
    """Signed floor(|v| 2^(86 - e)) for |v| < 2^e, exactly."""
    fr = Fraction(v) * Fraction(2) ** (86 - e)
    q = abs(fr.numerator) // fr.denominator
    return q if v >= 0 else -q


BIAS = sum(128 << (8 * i) for i in range(11))


def _digit(q: int, t: int) -> int:
    """Balanced digit t (1..11) of the image q: byte 11 - t of q + BIAS, less 128."""
    u = ((q + BIAS) >> (8 * (11 - t))) & 255
    return u - 128


def _digit_update(X, D, s):
    """X D with s balanced 8-bit digits per operand, as exact Fractions."""
    ce = _exps(X).max(axis=0)
    Xh = np.ldexp(X, -ce[None, :])
    r = _exps(Xh).max(axis=1)
    Dp = np.ldexp(D, ce[:, None])
    w = _exps(Dp).max(axis=0)
    qx = [[_fixed(float(Xh[l, a]), int(r[l])) for a in range(X.shape[1])] for l in range(X.shape[0])]
    qd = [[_fixed(float(Dp[a, j]), int(w[j])) for j in range(D.shape[1])] for a in range(D.shape[0])]
    dx = [np.array([[_digit(q, t) for q in row] for row in qx], dtype=object) for t in range(1, s + 1)]
    dd = [np.array([[_digit(q, t) for q in row] for row in qd], dtype=object) for t in range(1, s + 1)]
    acc = np.zeros((X.shape[0], D.shape[1]), dtype=object)
    for t in range(1, s + 1):
        for u in range(1, s + 2 - t):
            acc = acc + dx[t - 1].dot(dd[u - 1]) * (1 << (8 * (2 * s - t - u)))
    out = np.empty(acc.shape, dtype=object)
    for (l, j), v in np.ndenumerate(acc):
        # v = 2^(16 s) sum_(t+u<=s+1) d_t d_u 2^(-8 (t + u)); x = 2^(e + 2) sum d_t 2^(-8 t)
        out[l, j] = Fraction(int(v)) * Fraction(2) ** (int(r[l]) + int(w[j]) + 4 - 16 * s)
    return out


def test_balanced_digits_rebuild_the_image():
    """The balanced digits of an image add back up to it (the representation
    the kernels rely on), for extreme and random images."""
    rng = np.random.default_rng(5)
    cases = [0, 1, -1, 2 ** 86 - 1, -(2 ** 86 - 1), 2 ** 85, -(2 ** 85)]
    cases += [int(v) for v in rng.integers(-2 ** 62, 2 ** 62, size=50)]
    cases += [int(v) << 24 for v in rng.integers(-2 ** 61, 2 ** 61, size=50)]
    for q in cases:
        ds = [_digit(q, t) for t in range(1, 12)]
        assert all(-128 <= d <= 127 for d in ds)
        assert sum(d << (8 * (11 - t)) for t, d in enumerate(ds, start=1)) == q


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


def test_seven_digits_miss_fp64_accuracy_on_graded_iterates(graded_pivot):
    """A 56-bit update (7 digits per operand) exceeds FP64's per-entry bound on
    a large share of the entries: one exponent per row and column is not
    enough at that length on graded iterates."""
    ratio = _ratio(graded_pivot, 7)
    assert np.mean(ratio > 1) > 0.05 and np.max(ratio) > 100


def test_eleven_digits_meet_fp64_accuracy_on_graded_iterates(graded_pivot):
    """With 11 digits per operand (88 bits), the update's default, every
    entry is within FP64's bound with a wide margin."""
    ratio = _ratio(graded_pivot, 11)
    assert np.max(ratio) <= 0.05


def _kernel_fold(S, s=11, pa=6):
    """The update kernels' combination of the diagonal sums S[d] (d = 2..s+1):
    phase A folds the groups 2..pa+1, phase B the groups pa+2..s+1, each as
    Horner sums in base 256 with a pair of groups (d, d + 1) first combined in
    int32 when d <= 8, and the total is T = accA 256^(s - pa) + accB. Returns T,
    checking every int32 and int64 intermediate against its range."""
    def fold(lo, hi):
        acc, d = 0, lo
        while d + 1 <= hi and d <= 8:
            pr = S[d] * 256 + S[d + 1]
            assert -2 ** 31 <= pr < 2 ** 31
            acc = acc * 65536 + pr
            assert -2 ** 63 <= acc < 2 ** 63
            d += 2
        while d <= hi:
            acc = acc * 256 + S[d]
            assert -2 ** 63 <= acc < 2 ** 63
            d += 1
        return acc
    acc_a = fold(2, pa + 1)
    acc_b = fold(pa + 2, s + 1)
    return (acc_a << (8 * (s - pa))) + acc_b


def test_kernel_fold_order_gives_the_exact_digit_sum():
    """The kernels' fold of the group sums (int32 pairs, int64 Horner, the
    phase-A sum shifted by 8 (s - 6) bits) equals the plain sum
    sum_d S_d 256^(s + 1 - d), on random group sums and on the extreme ones
    (every digit -128, the largest magnitude a group can reach: d - 1
    products of 64 terms of 2^14)."""
    rng = np.random.default_rng(9)
    s = 11
    for trial in range(200):
        if trial == 0:
            S = {d: (d - 1) * 64 * 128 * 128 for d in range(2, s + 2)}
        elif trial == 1:
            S = {d: -(d - 1) * 64 * 128 * 128 for d in range(2, s + 2)}
        else:
            S = {d: int(rng.integers(-(d - 1) * 64 * 2 ** 14, (d - 1) * 64 * 2 ** 14 + 1))
                 for d in range(2, s + 2)}
        assert all(abs(v) < 2 ** 24 for v in S.values())  # exact in the fp32 accumulators
        ref = sum(S[d] * 256 ** (s + 1 - d) for d in range(2, s + 2))
        assert _kernel_fold(S, s) == ref
