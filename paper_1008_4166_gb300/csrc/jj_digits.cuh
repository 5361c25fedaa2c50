// Digits of the split-precision block update (2.9): fixed-point images cut
// into up to eleven balanced 8-bit digits (88 bits) per operand, and the
// W-side operand of the update built from W_P.
//
// Balanced digits. For |x| < 2^e the signed integer V = +-floor(|x| 2^(86-e))
// (|V| < 2^86, two's complement) plus the bias B = sum_{i=0..10} 128 * 256^i
// is a non-negative 88-bit number U whose bytes u_i give V = sum (u_i - 128)
// 256^i. Digit t (1..11) is d_t = u_(11-t) - 128 in [-128, 127], so that
//     x = 2^(e+2) sum_t d_t 2^(-8t) + r,   |r| < 2^(e-86).
// A digit is exact in fp16: the bit pattern 0x6500 + u is 1280 + u, and one
// f16x2 addition of -1408 leaves u - 128 in each half.
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

// The biased image U = V + B of x relative to 2^e (|x| < 2^e), 96 bits
// (the top byte is zero). Integer operations on the significand only; zeros
// and subnormals give V = 0.
__device__ __forceinline__ unsigned __int128 dg_image88(double x, int e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    unsigned __int128 M = 0;
    if (E != 0) {
        const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = E - 989 - e;  // V = mant 2^sh, sh <= 33 because |x| < 2^e
        if (sh >= 0)
            M = (unsigned __int128)mant << sh;
        else if (sh > -64)
            M = mant >> (-sh);
    }
    if ((long long)b < 0) M = (unsigned __int128)0 - M;
    const unsigned __int128 B = ((unsigned __int128)0x808080u << 64) |
                                (unsigned __int128)0x8080808080808080ull;
    return M + B;
}

// The same image as three 32-bit words (w0 the least significant), built with
// 32-bit funnel shifts and selects only (no branch, no 128-bit arithmetic):
// the significand, left-aligned in a 96-bit word, is shifted right by
// t = 43 - sh words and bits.
struct Img96 {
    uint32_t w0, w1, w2;
};
__device__ __forceinline__ Img96 dg_image96(double x, int e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
    const int E = (int)((bh >> 20) & 0x7FFu);
    const uint32_t z2 = __funnelshift_l(bl, bh, 11) | 0x80000000u;  // significand bits 52..21
    const uint32_t z1 = bl << 11;                                      // bits 20..0, then zeros
    // V = significand 2^(E - 1075 + 86 - e) = (z2:z1:0) >> t, t >= 10
    int t = 1032 - E + e;
    t = (E == 0 || t > 127) ? 127 : t;  // zeros and subnormals: V = 0
    const uint32_t q = (uint32_t)t >> 5, r = (uint32_t)t & 31u;
    const uint32_t c2 = z2 >> r;
    const uint32_t c1 = __funnelshift_r(z1, z2, r);
    const uint32_t c0 = __funnelshift_r(0u, z1, r);
    uint32_t w2 = q == 0 ? c2 : 0u;
    uint32_t w1 = q == 0 ? c1 : (q == 1 ? c2 : 0u);
    uint32_t w0 = q == 0 ? c0 : (q == 1 ? c1 : (q == 2 ? c2 : 0u));
    // two's complement when negative: (w ^ m) - m over 96 bits
    const uint32_t m = (uint32_t)((int32_t)bh >> 31);
    unsigned long long lo = ((unsigned long long)w1 << 32) | w0;
    const bool lz = lo == 0ull;
    lo = (lo ^ (((unsigned long long)m << 32) | m)) + (unsigned long long)(m & 1u);
    w2 = (w2 ^ m) + ((m & 1u) && lz ? 1u : 0u);
    // plus the bias 0x80 in each of the bytes 0..10
    const unsigned long long lb = lo + 0x8080808080808080ull;
    w2 += 0x808080u + (lb < lo ? 1u : 0u);
    return Img96{(uint32_t)lb, (uint32_t)(lb >> 32), w2};
}

// Byte u of digit t (1..11) of an image.
__device__ __forceinline__ uint32_t dg_byte88(unsigned __int128 U, int t) {
    return (uint32_t)(U >> (8 * (11 - t))) & 255u;
}

// The 24-bit window of U holding the bytes of digits 3p + 1, 3p + 2, 3p + 3
// (bits [64 - 24p, 88 - 24p), zero below bit 0): digit 3p + 1 + i has byte
// (window >> (16 - 8i)) & 255.
__device__ __forceinline__ uint32_t dg_window24(double x, int e, int p) {
    const unsigned __int128 U = dg_image88(x, e);
    const int sh = 64 - 24 * p;
    return (uint32_t)(sh >= 0 ? (U >> sh) : (U << (-sh))) & 0xFFFFFFu;
}

// Two digits given by their bytes u0, u1 as packed fp16 (u - 128 each).
__device__ __forceinline__ uint32_t dg_pack2(uint32_t u0, uint32_t u1) {
    const uint32_t v = u0 | (u1 << 16) | 0x65006500u;
    uint32_t r;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(0xE580E580u));
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
        const unsigned __int128 U0 = dg_image88(x0, s_wexp[j] - xexp[a]);
        const unsigned __int128 U1 = dg_image88(x1, s_wexp[j] - xexp[a + 1]);
        const uint32_t off = tc::sw128_off(j, a * 2);
        for (int t = 1; t <= slices; ++t)
            *reinterpret_cast<uint32_t *>(img + (size_t)(t - 1) * kUpdSliceBytes + off) =
                dg_pack2(dg_byte88(U0, t), dg_byte88(U1, t));
    }
    for (int j = tid; j < kUdPositions; j += nthreads) wexp_out[j] = s_wexp[j];
}

}  // namespace jj
