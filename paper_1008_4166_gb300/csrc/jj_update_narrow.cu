// Block update (2.9) [G_i G_j] <- [G_i G_j] W_P of narrow pivots (up to 64
// real-form positions: b <= 16 complex or b <= 32 real columns per block) as
// exact digit products on the tcgen05 tensor cores, with the pivot rows fed
// by TMA.
//
// The arithmetic is that of jj_update_digits.cu: the correction form
// Y = X + X (W2 - I), balanced 8-bit digits of X (one exponent per row, after
// the column exponents) and of D' = D (W2 - I) (one exponent per column), the
// digit products of one diagonal d = t + u summed exactly in one fp32 TMEM
// group, the groups folded in integers, one rounding per output. Only the
// data movement differs.
//
// Pipeline (one persistent CTA per SM; a contiguous range of the active
// (pair, 128-row tile) work items; 16 warps):
//   * producer (warp 9): per item, two passes over the tile in four chunks of
//     32 rows; each chunk (both blocks of the pivot) arrives by two tiled TMA
//     copies (cp.async.bulk.tensor.2d, 8 KB each) into a ring of two
//     shared-memory slots. The warp also writes the item's column exponents
//     to a small shared table.
//   * builders (warps 10..15, two groups of three): group g takes the chunks
//     of slot g; a lane owns one row of the chunk, the three warps of the
//     group split its columns. Pass 0 finds each row's exponent (a partial
//     maximum per warp, combined through shared memory) and writes digits
//     1..6; pass 1 writes digits 7..s. A digit of a value is a byte of its
//     biased fixed-point image (jj_digits.cuh), so a digit pair costs one
//     byte permute, one logic op and one f16x2 add. Lanes visit their column
//     pairs in an order rotated by lane group, so that the 32 lanes of a
//     store hit different banks of the swizzled tile.
//   * one thread (warp 8) issues the products as in jj_update_digits.cu:
//     phase A forms the groups 2..7 from A_1..A_6, phase B the groups 8..s+1
//     from A_1..A_s, over a ring of 6 TMEM slots of 64 columns.
//   * epilogue (warps 0..7, a TMEM lane quadrant and an output half each)
//     drains each pair of groups into int64 Horner sums, parks the phase-A
//     sum in TMEM columns 384..511 (no round trip through memory), and ends
//     with Y = X + corr: the int128 sum rounded to FP64 without branches.
//
// Every wait is bounded (tc::mbar_wait); a wait that runs out sets an error
// flag, every role leaves its loop, and the teardown waits for the products
// and copies in flight before the TMEM is freed.
#include <cuda.h>

#include "jj_common.cuh"
#include "jj_digits.cuh"
#include "jj_tc.cuh"

namespace jj {
namespace {

using namespace tc;

constexpr int UN_M = 128;                 // rows per work item (MMA M, TMEM lanes)
constexpr int UN_ASLOTS = 6;              // A digit tiles resident (digits 1..6, then 7..11)
constexpr int UN_TSLOTS = 6;              // TMEM group slots of 64 columns (columns 0..383)
constexpr uint32_t UN_PARK_COL = 384;     // TMEM columns 384..511: the parked phase-A sums
constexpr int UN_EPI = 8;                 // epilogue warps 0..7
constexpr int UN_MMA = 8;                 // warp 8 issues the products
constexpr int UN_PROD = 9;                // warp 9 feeds the chunks
constexpr int UN_BLD0 = 10;               // builder warps 10..15
constexpr int UN_BLD = 6;
constexpr int UN_GRP = 3;                 // builder warps per group (one group per chunk slot)
constexpr int UN_THREADS = 16 * 32;
constexpr int UN_ATILE = UN_M * 128;      // 16 KB per A digit tile
constexpr int UN_PA = 6;                  // digits (= groups) of phase A
constexpr int UN_RING = 4;                // row-exponent and column-exponent rings (items)
constexpr int UN_CROWS = 32;              // rows per chunk
constexpr int UN_BOX_BYTES = 8192;        // one TMA box: 32 rows x 16 complex or 32 real columns
constexpr int UN_CHUNK_BYTES = 2 * UN_BOX_BYTES;

// Columns per block that one box covers (the narrow pivot's blocks fit).
template <bool CPLX>
__host__ __device__ constexpr int un_boxc() { return CPLX ? 16 : 32; }

struct UnShared {
    unsigned long long a_full[UN_ASLOTS], a_empty[UN_ASLOTS];
    unsigned long long t_full[UN_TSLOTS], t_empty[UN_TSLOTS];
    unsigned long long x_full[2], x_empty[2];
    unsigned long long r_full[UN_RING], r_empty[UN_RING];
    unsigned long long b_full, mma_done;
    int rexp[UN_RING][UN_M];              // row exponents of an item
    int cx[UN_RING][64];                  // column exponents of an item's pivot columns
    unsigned long long pm_bar[2][2];      // builder group g, chunk cc: the partial maxima are in
    int pmax[2][2][UN_GRP][64];           // partial row maxima: [item parity][cc][warp][group g rows]
    uint32_t tmem_base;
    int abort;
    int q0, r0, count;
};

__device__ __forceinline__ int un_tiles(const StepCtl &c, int q, int64_t m) {
    return (int)((pair_rows(c, q, m) + UN_M - 1) / UN_M);
}
__device__ __forceinline__ bool un_active(const StepCtl &c, int q, int64_t m) {
    return !pair_passthrough(c, q) && un_tiles(c, q, m) > 0;
}
__device__ __forceinline__ void un_next(const StepCtl &c, int npairs, int64_t m, int &q, int &r) {
    if (++r < un_tiles(c, q, m)) return;
    r = 0;
    do {
        ++q;
    } while (q < npairs && !un_active(c, q, m));
}
__device__ __forceinline__ int64_t un_gcol(const int32_t *pd, int c) {
    return c < pd[1] ? (int64_t)pd[0] + c : (int64_t)pd[2] + (c - pd[1]);
}

// 32 lanes x 16 consecutive 32-bit TMEM columns: store and load.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// Out of the normal range (never for the method's inputs): ldexp, kept out of
// line so that the common path carries none of its instructions.
__device__ __noinline__ double un_scaled_slow(double d, int sc, bool neg) {
    const double v = ldexp(d, sc);
    return neg ? -v : v;
}

// (hi:lo), a two's-complement 128-bit integer, times 2^e rounded to the
// nearest double (ties to even). The magnitude is normalised so that its
// leading one is bit 63 of a 64-bit word t64 whose bit 0 also carries the OR
// of every bit below it (a sticky bit far under the rounding position); one
// correctly rounded conversion of t64 then rounds the whole value, and the
// power of two enters through the exponent field. Selects instead of
// branches: every lane of a warp takes the same instructions.
__device__ __forceinline__ double un_i128_to_double(long long hi, unsigned long long lo, int e) {
    const unsigned long long sg = (unsigned long long)(hi >> 63);  // all ones when negative
    unsigned long long l = lo ^ sg, h = (unsigned long long)hi ^ sg;
    const unsigned long long l2 = l - sg;  // + 1 when negative
    h += (l2 < l) ? 1ull : 0ull;
    l = l2;
    const bool hz = h == 0ull;
    const unsigned long long hs = hz ? l : h;  // the word with the leading one
    const unsigned long long ls = hz ? 0ull : l;
    const int z = __clzll((long long)hs);      // 64 when the value is zero
    const int zs = z & 63;
    const unsigned long long top = (hs << zs) | ((ls >> 1) >> (63 - zs));
    const unsigned long long t64 = top | ((ls << zs) != 0ull ? 1ull : 0ull);
    const int sc = e + 64 - ((hz ? 64 : 0) + z);  // |value| = t64 2^sc
    const double d = __ull2double_rn(t64);
    const long long bits = __double_as_longlong(d);
    const int ex = (int)((bits >> 52) & 0x7FF) + sc;
    if (hs == 0ull) return 0.0;
    if (__builtin_expect(ex < 1 || ex > 2046, 0)) return un_scaled_slow(d, sc, sg != 0ull);
    return __longlong_as_double(
        (long long)(((unsigned long long)bits + ((unsigned long long)(long long)sc << 52)) | (sg << 63)));
}

// Digits T0 .. T0 + NT - 1 (those up to t_hi) of two values at positions
// (a, a + 1) of one row: a 32-bit store per digit tile.
template <int T0, int NT>
__device__ __forceinline__ void un_store_digits(uint8_t *sA, uint32_t off, const Img96 &U0, const Img96 &U1,
                                                int t_hi) {
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        const int t = T0 + i;
        if (t > t_hi) break;
        const int kb = 11 - t, wi = kb >> 2, bi = kb & 3;
        const uint32_t w0 = wi == 0 ? U0.w0 : (wi == 1 ? U0.w1 : U0.w2);
        const uint32_t w1 = wi == 0 ? U1.w0 : (wi == 1 ? U1.w1 : U1.w2);
        const uint32_t v = (__byte_perm(w0, w1, (uint32_t)(bi | ((4 + bi) << 8))) & 0x00FF00FFu) | 0x65006500u;
        uint32_t h2;
        asm("add.rn.f16x2 %0, %1, %2;" : "=r"(h2) : "r"(v), "r"(0xE580E580u));
        *reinterpret_cast<uint32_t *>(sA + (size_t)((t - 1) % UN_ASLOTS) * UN_ATILE + off) = h2;
    }
}

template <bool CPLX, int NS>
__global__ void __launch_bounds__(UN_THREADS, 1) update_narrow_kernel(
    const __grid_constant__ CUtensorMap xmap, const double *Gs, double *Gd, int64_t ld, int64_t m,
    const int32_t *__restrict__ pairs, int npairs, const int32_t *__restrict__ cexp,
    const uint8_t *__restrict__ wimg, const int32_t *__restrict__ wexp, int slices,
    unsigned long long *__restrict__ counters, uint64_t wait_ns, StepCtl ctl) {
    constexpr int s = NS;  // digits per operand
    extern __shared__ __align__(1024) uint8_t un_smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>(((uintptr_t)un_smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sB = sm;                                    // s tiles of 8 KB (digits of D')
    uint8_t *sA = sm + (size_t)s * kUpdSliceBytes;       // 6 slots of 16 KB (digits of Xh)
    uint8_t *sX = sA + (size_t)UN_ASLOTS * UN_ATILE;     // 2 chunk slots of 16 KB (rows of X)
    __shared__ UnShared S;
    volatile int *abort_flag = &S.abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int hA = s < UN_PA ? s : UN_PA;  // digits (= groups) of phase A
    constexpr bool phaseB = s > UN_PA;
    constexpr int UPI = phaseB ? 8 : 4;        // chunk units per item (passes x 4 chunks)
    constexpr int E = CPLX ? 2 : 1;
    constexpr int BOXC = un_boxc<CPLX>();

    // ---- set-up: barriers, TMEM, this CTA's range of work items ----
    if (warp == UN_MMA) {
        tmem_alloc(su32(&S.tmem_base), 512);
        if (lane == 0) {
            for (int i = 0; i < UN_ASLOTS; ++i) {
                mbar_init(su32(&S.a_full[i]), 2 * UN_BLD);  // every builder warp, two chunks each
                mbar_init(su32(&S.a_empty[i]), 1);
            }
            for (int i = 0; i < UN_TSLOTS; ++i) {
                mbar_init(su32(&S.t_full[i]), 1);
                mbar_init(su32(&S.t_empty[i]), UN_EPI);
            }
            for (int i = 0; i < 2; ++i) {
                mbar_init(su32(&S.x_full[i]), 1);
                mbar_init(su32(&S.x_empty[i]), UN_GRP);
            }
            for (int i = 0; i < UN_RING; ++i) {
                mbar_init(su32(&S.r_full[i]), 4);  // one per chunk
                mbar_init(su32(&S.r_empty[i]), UN_EPI);
            }
            for (int i = 0; i < 4; ++i) mbar_init(su32(&S.pm_bar[i >> 1][i & 1]), UN_GRP * 32);
            mbar_init(su32(&S.b_full), 1);
            mbar_init(su32(&S.mma_done), 1);
            mbar_init_fence();
            S.abort = 0;
        }
        long long total = 0;
        for (int base = 0; base < npairs; base += 32) {
            const int q = base + lane;
            int t = (q < npairs && un_active(ctl, q, m)) ? un_tiles(ctl, q, m) : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            total += t;
        }
        const long long beg = total * blockIdx.x / gridDim.x;
        const long long end = total * (blockIdx.x + 1) / gridDim.x;
        long long acc = 0;
        int q0 = npairs, r0 = 0;
        for (int base = 0; base < npairs && q0 == npairs; base += 32) {
            const int q = base + lane;
            const int t = (q < npairs && un_active(ctl, q, m)) ? un_tiles(ctl, q, m) : 0;
            int inc = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            const long long lo = acc + inc - t;
            const unsigned hit = __ballot_sync(0xffffffffu, t > 0 && lo <= beg && beg < lo + t);
            if (hit) {
                const int src = __ffs(hit) - 1;
                q0 = __shfl_sync(0xffffffffu, q, src);
                r0 = (int)__shfl_sync(0xffffffffu, (int)(beg - lo), src);
            }
            acc += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) {
            S.q0 = q0;
            S.r0 = r0;
            S.count = beg < end ? (int)(end - beg) : 0;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    const int count = S.count;

    if (warp < UN_EPI) {
        // ------------------------------------------------------------------
        // Epilogue: thread = output row (TMEM lane), 32 output positions.
        // ------------------------------------------------------------------
        const int quad = warp & 3, hh = warp >> 2;
        const int rl = quad * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        int q = S.q0, r = S.r0;
        long long acc[32];
        // Fold N = 1 or 2 consecutive groups g (and g + 1) into the Horner sums
        // (int64, base 256: acc <- acc 256^N + sum). Group d holds at most d - 1
        // products, |S_d| <= (d - 1) 2^20, so a pair with d <= 8 folds in int32
        // first (|S_d 256 + S_(d+1)| <= 1800 * 2^20 < 2^31). The TMEM slots are
        // released after the fold. False when a wait ran out.
        auto wait_group = [&](long long gi) -> bool {
            const int slot = (int)(gi % UN_TSLOTS);
            const uint32_t par = (uint32_t)((gi / UN_TSLOTS) & 1);
            const bool ok = __all_sync(0xffffffffu, !*abort_flag && mbar_wait(su32(&S.t_full[slot]), par, wait_ns));
            if (!ok) *abort_flag = 1;
            return ok;
        };
        auto drain2 = [&](long long g) -> bool {
            if (!wait_group(g) || !wait_group(g + 1)) return false;
            tc_fence_after();
            const int s0 = (int)(g % UN_TSLOTS), s1 = (int)((g + 1) % UN_TSLOTS);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                uint32_t v0[8], v1[8];
                tmem_ld8(lane_base + (uint32_t)(s0 * 64 + hh * 32 + h * 8), v0);
                tmem_ld8(lane_base + (uint32_t)(s1 * 64 + hh * 32 + h * 8), v1);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int pr = __float2int_rn(__uint_as_float(v0[c])) * 256 + __float2int_rn(__uint_as_float(v1[c]));
                    acc[h * 8 + c] = acc[h * 8 + c] * 65536 + pr;  // exact integers
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(su32(&S.t_empty[s0]));
                mbar_arrive(su32(&S.t_empty[s1]));
            }
            return true;
        };
        auto drain1 = [&](long long g) -> bool {
            if (!wait_group(g)) return false;
            tc_fence_after();
            const int s0 = (int)(g % UN_TSLOTS);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                uint32_t v0[8];
                tmem_ld8(lane_base + (uint32_t)(s0 * 64 + hh * 32 + h * 8), v0);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    acc[h * 8 + c] = acc[h * 8 + c] * 256 + __float2int_rn(__uint_as_float(v0[c]));
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(su32(&S.t_empty[s0]));
            return true;
        };
        // groups [d_lo, d_hi] of an item, from zero sums
        auto drain_range = [&](long long g0, int d_lo, int d_hi) -> bool {
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = 0;
            int d = d_lo;
#pragma unroll 1
            for (; d + 1 <= d_hi && d <= 8; d += 2)
                if (!drain2(g0 + d - 2)) return false;
#pragma unroll 1
            for (; d <= d_hi; ++d)
                if (!drain1(g0 + d - 2)) return false;
            return true;
        };
        const uint32_t park = lane_base + UN_PARK_COL + (uint32_t)(hh * 64);
        for (int J = 0; J < count; ++J) {
            if (*abort_flag) break;
            const int32_t *pd = pairs + 4 * q;
            const int k = pd[1] + pd[3];
            const int64_t rows = pair_rows(ctl, q, m);
            const int64_t l = (int64_t)r * UN_M + rl;
            const long long g0 = (long long)J * s;
            if (!drain_range(g0, 2, hA + 1)) break;
            if (phaseB) {
                // park the phase-A sums (64 words: lo, hi of each output) in TMEM
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    uint32_t w[16];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        w[2 * c] = (uint32_t)(unsigned long long)acc[8 * b + c];
                        w[2 * c + 1] = (uint32_t)((unsigned long long)acc[8 * b + c] >> 32);
                    }
                    tmem_st16(park + (uint32_t)(16 * b), w);
                }
                tmem_wait_st();
                if (!drain_range(g0, UN_PA + 2, s + 1)) break;
            }
            const int rho = J % UN_RING;
            if (!__all_sync(0xffffffffu, mbar_wait(su32(&S.r_full[rho]), (uint32_t)((J / UN_RING) & 1), wait_ns))) {
                *abort_flag = 1;
                break;
            }
            const int re = S.rexp[rho][rl];
            // output position hh * 32 + c: pivot column c of part hh (complex), column
            // hh * 32 + c (real); element offsets of the row in the two blocks
            const int n1 = pd[1];
            const int64_t ldE = ld * E;
            const int64_t off_i = ((int64_t)pd[0] * ld + l) * E + (CPLX ? hh : 0);
            const int64_t off_j = ((int64_t)pd[2] * ld + l) * E + (CPLX ? hh : 0) - (int64_t)n1 * ldE;
            const int pc0 = CPLX ? 0 : hh * 32;
            const int4 *wx4 = reinterpret_cast<const int4 *>(wexp + (size_t)q * kUdPositions + hh * 32);
            constexpr int SH = 8 * (s - UN_PA);  // T = accA 2^(8 (s - 6)) + accB
            const int ebase = re + 4 - 8 * (s + 1);
            const bool row_ok = l < rows;
            tc_fence_after();
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                uint32_t w[8];
                if (phaseB) {
                    tmem_ld8(park + (uint32_t)(8 * b), w);
                    tmem_wait_ld();
                }
                const int4 w4 = wx4[b];
                const int wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int hp = 0; hp < 2; ++hp) {  // two outputs at a time (register pressure)
                    int64_t off[2];
                    bool in[2];
                    double xv[2];
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int pc = pc0 + 4 * b + 2 * hp + c;
                        in[c] = row_ok && pc < k;
                        off[c] = (pc < n1 ? off_i : off_j) + (int64_t)pc * ldE;
                        xv[c] = in[c] ? Gs[off[c]] : 0.0;
                    }
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int cc = 2 * hp + c;
                        const long long bb = acc[4 * b + cc];
                        long long hi;
                        unsigned long long lo;
                        if (phaseB) {
                            const long long a = (long long)(((unsigned long long)w[2 * cc + 1] << 32) | w[2 * cc]);
                            const unsigned long long al = (unsigned long long)a << SH;
                            const long long ah = a >> (64 - SH);
                            lo = al + (unsigned long long)bb;
                            hi = ah + (bb >> 63) + (lo < al ? 1 : 0);
                        } else {
                            lo = (unsigned long long)bb;
                            hi = bb >> 63;
                        }
                        const double y = xv[c] + un_i128_to_double(hi, lo, ebase + wv[cc]);
                        if (in[c]) Gd[off[c]] = y;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(su32(&S.r_empty[rho]));
            un_next(ctl, npairs, m, q, r);
        }
    } else if (warp == UN_MMA) {
        // ------------------------------------------------------------------
        // Product issue (one thread).
        // ------------------------------------------------------------------
        if (lane == 0) {
            int q = S.q0, r = S.r0;
            int prev_q = -1;
            uint32_t bpar = 0, dpar = 0;
            // a bulk copy / a commit whose completion has not been seen yet
            bool b_pending = false, d_pending = false;
            const uint32_t a_base = su32(sA), b_base = su32(sB);
            bool ok = true;
            auto waitb = [&](unsigned long long *bar, uint32_t par) {
                if (ok && (*abort_flag || !mbar_wait(su32(bar), par, wait_ns))) {
                    ok = false;
                    *abort_flag = 1;
                }
            };
            // products A_t x B_u for u in [u_lo, u_hi] into the groups t + u
            auto issue = [&](long long g0, int t, int u_lo, int u_hi) {
                const uint32_t a0 = a_base + (uint32_t)(((t - 1) % UN_ASLOTS) * UN_ATILE);
                for (int u = u_lo; u <= u_hi;) {
                    const long long g = g0 + t + u - 2;
                    const int slot = (int)(g % UN_TSLOTS);
                    int run = u_hi - u + 1;
                    run = min(run, 4);
                    run = min(run, UN_TSLOTS - slot);
                    const uint32_t id = idesc_f16(UN_M, 64 * run);
                    const uint32_t b0 = b_base + (uint32_t)((u - 1) * kUpdSliceBytes);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        mma_f16(tmem + (uint32_t)(slot * 64), desc_sw128(a0 + ks * 32),
                                desc_sw128(b0 + ks * 32), id, (t == 1 && ks == 0) ? 0u : 1u);
                    u += run;
                }
            };
            // before the first product of groups [d_lo, d_hi]: their TMEM slots
            // have been drained by the epilogue
            auto wait_slots = [&](long long g0, int d_lo, int d_hi) {
                for (int d = d_lo; d <= d_hi; ++d) {
                    const long long g = g0 + d - 2;
                    if (g >= UN_TSLOTS) waitb(&S.t_empty[g % UN_TSLOTS], (uint32_t)(((g / UN_TSLOTS) - 1) & 1));
                }
            };
            for (int J = 0; J < count && ok; ++J) {
                if (q != prev_q) {
                    // the digits of the new pair's D', once the products reading the old ones are done
                    if (prev_q >= 0) {
                        mma_commit(su32(&S.mma_done));
                        d_pending = true;
                        waitb(&S.mma_done, dpar);
                        if (!ok) break;
                        d_pending = false;
                        dpar ^= 1u;
                    }
                    mbar_expect_tx(su32(&S.b_full), (uint32_t)(s * kUpdSliceBytes));
                    bulk_g2s(b_base, wimg + (size_t)q * slices * kUpdSliceBytes, (uint32_t)(s * kUpdSliceBytes),
                             su32(&S.b_full));
                    b_pending = true;
                    waitb(&S.b_full, bpar);
                    if (!ok) break;
                    b_pending = false;
                    bpar ^= 1u;
                    prev_q = q;
                }
                const long long g0 = (long long)J * s;
                // phase A: groups 2..hA+1 from A_1..A_hA
                for (int t = 1; t <= hA && ok; ++t) {
                    const int sl = t - 1;
                    const int nuse = (sl + UN_PA + 1 <= s) ? 2 : 1;
                    waitb(&S.a_full[sl], (uint32_t)((J * nuse) & 1));
                    if (t == 1) wait_slots(g0, 2, hA + 1);
                    if (!ok) break;
                    tc_fence_after();
                    issue(g0, t, 1, hA + 1 - t);
                    mma_commit(su32(&S.t_full[(g0 + t - 1) % UN_TSLOTS]));  // group t + 1 is complete
                    if (!phaseB) mma_commit(su32(&S.a_empty[sl]));
                }
                // phase B: groups 8..s+1 from A_1..A_s
                for (int t = 1; phaseB && t <= s && ok; ++t) {
                    const int sl = (t - 1) % UN_ASLOTS;
                    if (t > UN_PA) waitb(&S.a_full[sl], (uint32_t)((J * 2 + 1) & 1));
                    if (t == 1) wait_slots(g0, UN_PA + 2, s + 1);
                    if (!ok) break;
                    tc_fence_after();
                    issue(g0, t, max(1, UN_PA + 2 - t), s + 1 - t);
                    mma_commit(su32(&S.a_empty[sl]));
                    if (t + 1 >= UN_PA + 2) mma_commit(su32(&S.t_full[(g0 + t - 1) % UN_TSLOTS]));
                }
                un_next(ctl, npairs, m, q, r);
            }
            // every product and copy has completed before the TMEM and the shared
            // memory are released
            if (!d_pending) mma_commit(su32(&S.mma_done));
            if (!mbar_wait(su32(&S.mma_done), dpar, kWaitLimitNs)) *abort_flag = 1;
            if (b_pending && !mbar_wait(su32(&S.b_full), bpar, kWaitLimitNs)) *abort_flag = 1;
        }
    } else if (warp == UN_PROD) {
        // ------------------------------------------------------------------
        // Producer: the column exponents of each item, and its rows by TMA.
        // ------------------------------------------------------------------
        int q = S.q0, r = S.r0;
        bool ok = true;
        long long last[2] = {-1, -1};  // last chunk unit issued into each slot
        const uint32_t x_base = su32(sX);
        for (int J = 0; J < count && ok; ++J) {
            const int32_t *pd = pairs + 4 * q;
            const int k = pd[1] + pd[3];
            for (int p = 0; p < UPI / 4 && ok; ++p) {
                for (int c = 0; c < 4 && ok; ++c) {
                    const long long U = (long long)J * UPI + p * 4 + c;
                    const int slot = (int)(U & 1);
                    if (U >= 2 &&
                        !__all_sync(0xffffffffu, !*abort_flag && mbar_wait(su32(&S.x_empty[slot]),
                                                                          (uint32_t)(((U >> 1) - 1) & 1), wait_ns))) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    if (p == 0 && c == 0) {
                        // the builders of item J - 2 and earlier are done: the
                        // table of item J - UN_RING is free
                        int *cx = S.cx[J % UN_RING];
                        for (int pc = lane; pc < 64; pc += 32) cx[pc] = pc < k ? cexp[un_gcol(pd, pc)] : -1021;
                    }
                    __syncwarp();
                    if (lane == 0) {
                        const uint32_t bar = su32(&S.x_full[slot]);
                        const uint32_t dst = x_base + (uint32_t)(slot * UN_CHUNK_BYTES);
                        const int y = E * (r * UN_M + c * UN_CROWS);
                        mbar_expect_tx(bar, (uint32_t)(((pd[1] > 0) + (pd[3] > 0)) * UN_BOX_BYTES));
                        if (pd[1] > 0) tma_load_2d(dst, &xmap, y, pd[0], bar);
                        if (pd[3] > 0) tma_load_2d(dst + UN_BOX_BYTES, &xmap, y, pd[2], bar);
                    }
                    last[slot] = U;
                }
            }
            un_next(ctl, npairs, m, q, r);
        }
        // the copies in flight land before the shared memory is released
        if (lane == 0)
            for (int sl = 0; sl < 2; ++sl)
                if (last[sl] >= 0 && !mbar_wait(su32(&S.x_full[sl]), (uint32_t)((last[sl] >> 1) & 1), kWaitLimitNs))
                    *abort_flag = 1;
    } else if (warp >= UN_BLD0) {
        // ------------------------------------------------------------------
        // Builders: digits of Xh = X D^-1 relative to each row's exponent.
        // ------------------------------------------------------------------
        const int bw = warp - UN_BLD0, g = bw / UN_GRP, mi = bw % UN_GRP;
        const int lg = lane >> 3;
        constexpr int NCP = CPLX ? 16 : 32;                      // column pairs of the pivot
        const int ncp = (NCP - mi + UN_GRP - 1) / UN_GRP;         // this warp's: mi, mi + 3, ...
        constexpr int CSTRIDE = CPLX ? 512 : 256;                // bytes per column of a box
        int q = S.q0, r = S.r0;
        bool ok = true;
        auto waitb = [&](unsigned long long *bar, uint32_t par) {
            if (!ok) return;
            if (!__all_sync(0xffffffffu, !*abort_flag && mbar_wait(su32(bar), par, wait_ns))) {
                ok = false;
                *abort_flag = 1;
            }
        };
        for (int J = 0; J < count && ok; ++J) {
            const int32_t *pd = pairs + 4 * q;
            const int k = pd[1] + pd[3], n1 = pd[1];
            const int rho = J % UN_RING;
            const int *cx = S.cx[rho];
            int rexp_c[2] = {-1021, -1021};
            for (int p = 0; p < UPI / 4 && ok; ++p) {
                for (int cc = 0; cc < 2 && ok; ++cc) {
                    const int c = g + 2 * cc;  // chunk of rows c * 32 ..
                    const long long U = (long long)J * UPI + p * 4 + c;
                    waitb(&S.x_full[g], (uint32_t)((U >> 1) & 1));
                    if (!ok) break;
                    const uint8_t *X = sX + (size_t)g * UN_CHUNK_BYTES;
                    auto col = [&](int pc) -> const uint8_t * {
                        return X + (size_t)(pc < n1 ? pc : BOXC + (pc - n1)) * CSTRIDE;
                    };
                    if (p == 0) {
                        // row exponent: max over the row of exp(x) - e_col
                        int mx = -100000;
                        for (int i = 0; i < ncp; ++i) {
                            const int pc0 = 2 * (mi + UN_GRP * i);
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int pc = pc0 + h;
                                if (pc >= k) continue;
                                if (CPLX) {
                                    const double2 z = reinterpret_cast<const double2 *>(col(pc))[lane];
                                    const unsigned long long a = dg_mag_bits(z.x), b = dg_mag_bits(z.y);
                                    const unsigned long long mb = a > b ? a : b;
                                    if (mb) mx = max(mx, dg_exp_of_bits(mb) - cx[pc]);
                                } else {
                                    const unsigned long long mb = dg_mag_bits(reinterpret_cast<const double *>(col(pc))[lane]);
                                    if (mb) mx = max(mx, dg_exp_of_bits(mb) - cx[pc]);
                                }
                            }
                        }
                        // combine the group's partial maxima (a bounded wait: a warp
                        // that left after a timeout makes the others time out too)
                        int (*pm)[64] = S.pmax[J & 1][cc];
                        pm[mi][lane + 32 * g] = mx;
                        mbar_arrive(su32(&S.pm_bar[g][cc]));
                        waitb(&S.pm_bar[g][cc], (uint32_t)(J & 1));
                        if (!ok) break;
                        mx = max(max(pm[0][lane + 32 * g], pm[1][lane + 32 * g]), pm[2][lane + 32 * g]);
                        rexp_c[cc] = mx == -100000 ? -1021 : mx;
                        if (mi == 0) {
                            if (cc == 0 && J >= UN_RING) waitb(&S.r_empty[rho], (uint32_t)(((J / UN_RING) - 1) & 1));
                            if (!ok) break;
                            S.rexp[rho][c * UN_CROWS + lane] = rexp_c[cc];
                            __syncwarp();
                            if (lane == 0) mbar_arrive(su32(&S.r_full[rho]));
                        }
                    }
                    const int rexp = rexp_c[cc];
                    // the slots of this pass's digits are free (once per item and pass)
                    const int t_lo = p == 0 ? 1 : UN_PA + 1, t_hi = p == 0 ? hA : s;
                    if (cc == 0) {
                        for (int t = t_lo; t <= t_hi; ++t) {
                            const int sl = (t - 1) % UN_ASLOTS;
                            const int nuse = (sl + UN_PA + 1 <= s) ? 2 : 1;
                            const long long f = (long long)J * nuse + (t > UN_PA ? 1 : 0);
                            if (f >= 1) waitb(&S.a_empty[sl], (uint32_t)((f - 1) & 1));
                        }
                        if (!ok) break;
                    }
                    const int row = c * UN_CROWS + lane;
                    for (int i = 0; i < ncp; ++i) {
                        // rotated by lane group: the lanes of one store hit different banks
                        int ii = i + lg;
                        ii -= ii >= ncp ? ncp : 0;
                        ii -= ii >= ncp ? ncp : 0;
                        ii -= ii >= ncp ? ncp : 0;
                        const int pc0 = 2 * (mi + UN_GRP * ii);
                        const bool in0 = pc0 < k, in1 = pc0 + 1 < k;
                        const int e0 = rexp + cx[pc0], e1 = rexp + cx[pc0 + 1];
                        if (CPLX) {
                            const double2 z0 = in0 ? reinterpret_cast<const double2 *>(col(pc0))[lane] : make_double2(0.0, 0.0);
                            const double2 z1 = in1 ? reinterpret_cast<const double2 *>(col(pc0 + 1))[lane] : make_double2(0.0, 0.0);
                            const Img96 R0 = dg_image96(z0.x, e0), R1 = dg_image96(z1.x, e1);
                            const Img96 I0 = dg_image96(z0.y, e0), I1 = dg_image96(z1.y, e1);
                            const uint32_t offr = sw128_off(row, pc0 * 2), offi = sw128_off(row, (32 + pc0) * 2);
                            if (p == 0) {
                                un_store_digits<1, UN_PA>(sA, offr, R0, R1, t_hi);
                                un_store_digits<1, UN_PA>(sA, offi, I0, I1, t_hi);
                            } else {
                                un_store_digits<UN_PA + 1, kUdMaxSlices - UN_PA>(sA, offr, R0, R1, t_hi);
                                un_store_digits<UN_PA + 1, kUdMaxSlices - UN_PA>(sA, offi, I0, I1, t_hi);
                            }
                        } else {
                            const double v0 = in0 ? reinterpret_cast<const double *>(col(pc0))[lane] : 0.0;
                            const double v1 = in1 ? reinterpret_cast<const double *>(col(pc0 + 1))[lane] : 0.0;
                            const Img96 U0 = dg_image96(v0, e0), U1 = dg_image96(v1, e1);
                            const uint32_t off = sw128_off(row, pc0 * 2);
                            if (p == 0)
                                un_store_digits<1, UN_PA>(sA, off, U0, U1, t_hi);
                            else
                                un_store_digits<UN_PA + 1, kUdMaxSlices - UN_PA>(sA, off, U0, U1, t_hi);
                        }
                    }
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(su32(&S.x_empty[g]));
                        for (int t = t_lo; t <= t_hi; ++t) mbar_arrive(su32(&S.a_full[(t - 1) % UN_ASLOTS]));
                    }
                }
            }
            un_next(ctl, npairs, m, q, r);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && S.abort && counters) atomicOr(&counters[kCntErr], kErrTimeout);
    if (warp == UN_MMA) tmem_dealloc(tmem, 512);
}

}  // namespace

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, found once (no link against libcuda).
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

}  // namespace

bool un_supported(bool cplx, const double *Gs, int64_t ld, int64_t m, int64_t ncols, int kmax, int maxblk) {
    const int E = cplx ? 2 : 1;
    if (ud_max_tiles(cplx, kmax) != 1) return false;
    if (maxblk < 0 || maxblk > (cplx ? un_boxc<true>() : un_boxc<false>())) return false;
    if (((uintptr_t)Gs & 15) != 0 || ((ld * E * 8) & 15) != 0) return false;
    if (m < 1 || ncols < 1 || (uint64_t)ld * E >= (1ull << 31) || ncols >= (1ll << 31)) return false;
    return encode_tiled() != nullptr;
}

bool encode_x_map(CUtensorMap *map, bool cplx, const double *G, int64_t ld, int64_t m, int64_t ncols,
                  int box_rows, int box_cols) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const int E = cplx ? 2 : 1;
    const cuuint64_t dims[2] = {(cuuint64_t)(m * E), (cuuint64_t)ncols};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * E * 8)};
    const cuuint32_t box[2] = {(cuuint32_t)(E * box_rows), (cuuint32_t)box_cols};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(G), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_update_narrow(bool cplx, const double *Gs, double *Gd, int64_t ld, int64_t m, int64_t ncols,
                                 const int32_t *pairs, int npairs, const int32_t *cexp, const UpdDigits &ud,
                                 int nctas, unsigned long long *counters, cudaStream_t st, StepCtl ctl) {
    const int s = ud.slices;
    if (s != kUdMaxSlices || !ud.img || !ud.wexp || nctas < 1) return cudaErrorInvalidValue;
    CUtensorMap map;
    if (!encode_x_map(&map, cplx, Gs, ld, m, ncols, UN_CROWS, cplx ? un_boxc<true>() : un_boxc<false>()))
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)s * kUpdSliceBytes + (size_t)UN_ASLOTS * UN_ATILE + 2 * (size_t)UN_CHUNK_BYTES + 1024;
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<nctas, UN_THREADS, smem, st>>>(map, Gs, Gd, ld, m, pairs, npairs, cexp, ud.img, ud.wexp, ud.slices,
                                              counters, ctl.wait_ns, ctl);
        return cudaGetLastError();
    };
    return cplx ? run(update_narrow_kernel<true, kUdMaxSlices>) : run(update_narrow_kernel<false, kUdMaxSlices>);
}

}  // namespace jj
