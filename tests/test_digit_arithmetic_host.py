"""The integer arithmetic of the split-precision update, compiled for the host
and checked against exact rational arithmetic (no GPU).

Two device routines decide the update's bits:
  * dg_image96 (csrc/jj_digits.cuh): the biased 88-bit fixed-point image of a
    double, V = +-floor(|x| 2^(86 - e)) plus 128 in each of the bytes 0..10,
    whose bytes give the balanced 8-bit digits;
  * un_i128_to_double (csrc/jj_update_narrow.cu): an int128 times 2^e rounded
    to the nearest double, ties to even.
The test lifts their source text out of the CUDA files, compiles it with g++
next to small stand-ins for the CUDA bit-cast and leading-zero intrinsics, and
compares the results with Python's exact integers and correctly rounded
Fraction -> float conversion on random, extreme and tie cases."""
import os
import random
import re
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1008_4166_gb300", "csrc")

SHIMS = r"""
#include <cstdint>
#include <cstring>
#include <cstdio>
#include <cmath>
#define __device__
#define __forceinline__ inline
#define __noinline__ __attribute__((noinline))
static inline long long __double_as_longlong(double x) { long long r; std::memcpy(&r, &x, 8); return r; }
static inline double __longlong_as_double(long long x) { double r; std::memcpy(&r, &x, 8); return r; }
static inline int __clzll(long long x) { return x == 0 ? 64 : __builtin_clzll((unsigned long long)x); }
static inline double __ull2double_rn(unsigned long long x) { return (double)x; }
static inline uint32_t __funnelshift_l(uint32_t lo, uint32_t hi, uint32_t s) {
    s &= 31; return (uint32_t)(((((uint64_t)hi << 32) | lo) << s) >> 32); }
static inline uint32_t __funnelshift_r(uint32_t lo, uint32_t hi, uint32_t s) {
    s &= 31; return (uint32_t)((((uint64_t)hi << 32) | lo) >> s); }
"""

MAIN = r"""
int main() {
    char op;
    while (std::scanf(" %c", &op) == 1) {
        if (op == 'I') {
            unsigned long long bits; int e;
            std::scanf("%llx %d", &bits, &e);
            double x; std::memcpy(&x, &bits, 8);
            Img96 w = dg_image96(x, e);
            std::printf("%08x%08x%08x\n", w.w2, w.w1, w.w0);
        } else {
            long long hi; unsigned long long lo; int e;
            std::scanf("%lld %llu %d", &hi, &lo, &e);
            std::printf("%016llx\n", (unsigned long long)__double_as_longlong(un_i128_to_double(hi, lo, e)));
        }
    }
    return 0;
}
"""


def _between(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def tool(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    digits = open(os.path.join(CSRC, "jj_digits.cuh")).read()
    narrow = open(os.path.join(CSRC, "jj_update_narrow.cu")).read()
    img = _between(digits, "struct Img96 {", "// Byte u of digit t")
    conv = _between(narrow, "__device__ __noinline__ double un_scaled_slow", "// Digits T0 .. T0 + NT - 1")
    d = tmp_path_factory.mktemp("digit_host")
    src = d / "t.cpp"
    src.write_text(SHIMS + img + conv + MAIN)
    exe = d / "t"
    subprocess.check_call(["g++", "-O1", "-std=c++17", str(src), "-o", str(exe)])

    def run(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout.split()
        assert len(out) == len(lines)
        return out
    return run


def _bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _exact_image(x: float, e: int) -> int:
    """V + bias for |x| < 2^e, V = sign(x) floor(|x| 2^(86 - e)), modulo 2^96."""
    q = abs(Fraction(x)) * Fraction(2) ** (86 - e)
    v = q.numerator // q.denominator
    if x < 0 or (x == 0 and struct.pack("<d", x)[7] & 0x80):
        v = -v
    return (v + sum(128 << (8 * i) for i in range(11))) % (1 << 96)


def test_digit_image_matches_exact_arithmetic(tool):
    rng = random.Random(3)
    cases = []
    for k in range(4000):
        m = rng.random()
        x = m * 2.0 ** rng.randint(-300, 300)
        if k % 2:
            x = -x
        if k % 97 == 0:
            x = 0.0
        fe = (abs(x).hex().split("p")[1] if x != 0 else "0")
        e0 = int(fe) + 1 if x != 0 else rng.randint(-50, 50)
        e = e0 if k % 3 == 0 else e0 + rng.randint(0, 120)  # tight and loose scales
        cases.append((x, e))
    cases += [(5e-324, 0), (-5e-324, 3), (2.0 ** -1022, -1021), (-(2.0 - 2.0 ** -52), 1)]
    out = tool(["I %x %d" % (_bits(x), e) for x, e in cases])
    for (x, e), got in zip(cases, out):
        u = int(got, 16)
        assert u == _exact_image(x, e), (x, e)
        # the balanced digits rebuild V
        ds = [((u >> (8 * (11 - t))) & 255) - 128 for t in range(1, 12)]
        v = sum(d << (8 * (11 - t)) for t, d in enumerate(ds, start=1))
        q = abs(Fraction(x)) * Fraction(2) ** (86 - e)
        assert abs(v) == q.numerator // q.denominator


def test_int128_rounding_is_correct_to_nearest_even(tool):
    rng = random.Random(4)
    cases = []
    for k in range(6000):
        nb = rng.randint(0, 101)
        t = rng.getrandbits(nb) if nb else 0
        if k % 5 == 0:  # exact ties at the rounding position of a 53-bit significand
            t = (rng.getrandbits(53) << 1 | 1) << rng.randint(0, 40) if nb > 60 else t
        if k % 2:
            t = -t
        cases.append((t, rng.randint(-200, 60)))
    cases += [(0, 5), (1, 0), (-1, 0), ((1 << 100) - 1, -100), (-(1 << 100), 3)]
    lines = []
    for t, e in cases:
        lo = t & ((1 << 64) - 1)
        hi = (t - lo) >> 64
        lines.append("C %d %d %d" % (hi, lo, e))
    out = tool(lines)
    for (t, e), got in zip(cases, out):
        ref = float(Fraction(t) * Fraction(2) ** e)
        assert int(got, 16) == _bits(ref) or (t == 0 and int(got, 16) in (0, 1 << 63)), (t, e)
