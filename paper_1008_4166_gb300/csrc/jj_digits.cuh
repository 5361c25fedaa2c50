// Digits of the split-precision block update (2.9): fixed-point images with
// up to twelve 7-bit digits (84 bits) per operand, and the W-side operand of
// the update built from W_P.
//
// Real-form positions of the update. A complex pivot X = Xr + i Xi with
// k <= 32 columns is handled as the real 64-position matrix whose position
// p < 32 holds Re of column p and position 32 + p holds Im of column p
// (positions of columns >= k are zero); a real pivot with k <= 64 columns
// takes position p = column p. The same positions index the rows (K) and the
// columns (N) of W2 = [[Wr, Wi], [-Wi, Wr]], so that [Yr | Yi] = [Xr | Xi] W2.
#pragma once

#include "jj_common.cuh"
#include "jj_tc.cuh"

namespace jj {

constexpr int kUdPositions = 64;  // real-form positions of a pivot

// V = floor(|x| 2^(84 - e)) for |x| < 2^e, as hi = V >> 20 (64 bits) and
// lo = V mod 2^21 (bit 20 is in both). Integer shifts of the significand
// only; zeros and subnormals give 0.
struct Fx84 {
    unsigned long long hi;
    uint32_t lo;
};
__device__ __forceinline__ Fx84 dg_fixed84(double x, int e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    Fx84 r{0ull, 0u};
    if (E == 0) return r;
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - 991 - e;  // V = mant 2^sh, and sh <= 31 because |x| < 2^e
    const int shh = sh - 20;
    if (shh >= 0)
        r.hi = mant << shh;  // shh <= 11: below 2^64
    else if (shh > -64)
        r.hi = mant >> (-shh);
    if (sh >= 0)
        r.lo = (uint32_t)((mant << sh) & 0x1FFFFFull);  // the low bits survive the wrap
    else if (sh > -64)
        r.lo = (uint32_t)((mant >> (-sh)) & 0x1FFFFFull);
    return r;
}

// 7-bit digit t (1..12) of V: bits [84 - 7t, 91 - 7t).
__device__ __forceinline__ uint32_t dg_digit84(const Fx84 &f, int t) {
    return t <= 9 ? (uint32_t)(f.hi >> (64 - 7 * t)) & 127u : (f.lo >> (84 - 7 * t)) & 127u;
}

// The 21-bit window of V = floor(|x| 2^(84 - e)) (|x| < 2^e) that holds the
// digits 3p + 1, 3p + 2, 3p + 3: bits [63 - 21p, 84 - 21p) of V, so that digit
// 3p + 1 + i is (window >> (14 - 7i)) & 127. Integer shifts only.
__device__ __forceinline__ uint32_t dg_window21(double x, int e, int p) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0) return 0u;
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - 1054 - e + 21 * p;  // V >> (63 - 21p) = mant 2^sh, sh <= 31
    unsigned long long w = 0ull;
    if (sh >= 0)
        w = mant << sh;  // only the low 21 bits are kept
    else if (sh > -64)
        w = mant >> (-sh);
    return (uint32_t)w & 0x1FFFFFu;
}

// Two signed digits as packed fp16 bits: +-d is (1024 + d) - 1024 in fp16 (the
// bit pattern of +-(1024 + d) is (0x6400 or 0xE400) | d; adding -+1024 leaves
// +-d exactly).
__device__ __forceinline__ uint32_t dg_pack2(uint32_t d0, bool n0, uint32_t d1, bool n1) {
    const uint32_t bias = (n0 ? 0xE400u : 0x6400u) | ((n1 ? 0xE400u : 0x6400u) << 16);
    const uint32_t add = bias ^ 0x80008000u;
    const uint32_t v = d0 | (d1 << 16) | bias;
    uint32_t r;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(add));
    return r;
}

// One 64 x 64 tile of W2 - delta I on real-form positions (a, j): the tile of
// row block kc and column block nc of a (possibly wide) pivot, w(r, c, part)
// returning part 0 (real) or 1 (imaginary) of W_P[r][c] relative to the
// tile's corner (complex: 32 pivot columns per tile, position p < 32 the real
// part of column p and 32 + p its imaginary part; real: 64 columns per tile).
// kr and kn: pivot columns present in the row and the column block; diag:
// the tile lies on the diagonal (kc = nc), where the identity is subtracted.
template <bool CPLX, typename WAcc>
__device__ __forceinline__ double ud_w2m(const WAcc &w, int kr, int kn, bool diag, int a, int j) {
    if (CPLX) {
        const int ra = a >> 5, ca = a & 31, rj = j >> 5, cj = j & 31;
        if (ca >= kr || cj >= kn) return 0.0;
        double v = ra == rj ? w(ca, cj, 0) : (ra == 0 ? w(ca, cj, 1) : -w(ca, cj, 1));
        return (diag && a == j) ? v - 1.0 : v;
    }
    if (a >= kr || j >= kn) return 0.0;
    const double v = w(a, j, 0);
    return (diag && a == j) ? v - 1.0 : v;
}

// The W-side operand of the digit update for one pair (one tile (kc, nc) of a
// wide pivot, as ud_w2m): the digits of D' = diag(2^e_a) (W2 - delta I),
// column j relative to its own exponent w_j
// (D'_aj < 2^w_j), as `slices` SWIZZLE_128B K-major tiles of 64 rows (row j =
// output position j) x 128 bytes (64 fp16 along K = position a), tile u at
// (u - 1) * kUpdSliceBytes, and the exponents w_j. The power-of-two scaling is
// exact (it moves the reference exponent of each digit, not the value).
// xexp[a]: column exponent e_a of position a (any value where the position is
// empty). Called by every thread of the block; s_wexp is 64 ints of shared
// memory.
template <bool CPLX, typename WAcc>
__device__ void ud_wimage_build(const WAcc &w, int kr, int kn, bool diag, const int *xexp, int *s_wexp,
                                int slices, uint8_t *img, int32_t *wexp_out, int tid, int nthreads) {
    const int warp = tid >> 5, lane = tid & 31, nw = nthreads >> 5;
    for (int j = warp; j < kUdPositions; j += nw) {
        int mx = -100000;
        for (int a = lane; a < kUdPositions; a += 32) {
            const unsigned long long mb = dg_mag_bits(ud_w2m<CPLX>(w, kr, kn, diag, a, j));
            if (mb) mx = max(mx, dg_exp_of_bits(mb) + xexp[a]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_wexp[j] = mx == -100000 ? -1021 : mx;
    }
    __syncthreads();
    for (int it = tid; it < kUdPositions * (kUdPositions / 2); it += nthreads) {
        const int j = it / (kUdPositions / 2), a = (it % (kUdPositions / 2)) * 2;
        const double x0 = ud_w2m<CPLX>(w, kr, kn, diag, a, j), x1 = ud_w2m<CPLX>(w, kr, kn, diag, a + 1, j);
        const Fx84 f0 = dg_fixed84(x0, s_wexp[j] - xexp[a]);
        const Fx84 f1 = dg_fixed84(x1, s_wexp[j] - xexp[a + 1]);
        const bool n0 = __double_as_longlong(x0) < 0, n1 = __double_as_longlong(x1) < 0;
        const uint32_t off = tc::sw128_off(j, a * 2);
        for (int t = 1; t <= slices; ++t)
            *reinterpret_cast<uint32_t *>(img + (size_t)(t - 1) * kUpdSliceBytes + off) =
                dg_pack2(dg_digit84(f0, t), n0, dg_digit84(f1, t), n1);
    }
    for (int j = tid; j < kUdPositions; j += nthreads) wexp_out[j] = s_wexp[j];
}

}  // namespace jj
