// Block update (2.9) [G_i G_j] <- [G_i G_j] W_P as exact digit products on
// the tcgen05 tensor cores, accurate to FP64's per-entry error on graded
// inputs.
//
// Correction form. Y = X W2 = X + X (W2 - I) on the real form X of the pivot
// (jj_digits.cuh): only the correction goes through digits, and the identity
// part is the exact FP64 entry of X.
//
// Scaling. X = Xh D with D = diag(2^e_a) the column exponents of the pivot
// columns; X (W2 - I) = Xh D'. The rows of Xh carry one exponent each (r_l)
// and the columns of D' = D (W2 - I) one each (w_j), so the digit products
// approximate
//     corr_lj = 2^(r_l + w_j + 4) sum_{t + u <= s + 1} 2^(-8 (t + u)) (Q_t P_u)_lj
// with Q_t, P_u the t-th and u-th balanced 8-bit digit matrices (digits in
// [-128, 127], exact in fp16; jj_digits.cuh) of Xh and D' relative to 2^r and
// 2^w. The error is relative to 2^(r_l + w_j), a row scale times a column
// scale; with s = 11 digits (88 bits) it stays below FP64's own per-entry
// bound u (|x_lj| + sum_a |x_la| |d_aj|) on the graded iterates of the method,
// where 56 bits exceed it by up to 7e5.
//
// Exactness. All products of one diagonal d = t + u share the weight 2^-8d
// and accumulate in one fp32 TMEM group: at most 11 products of K = 64 terms
// of at most 128^2 in magnitude, below 2^24, so every group sum is an exact
// integer. The groups are combined with integer shifts (Horner in int64), and
// one rounding to FP64 ends each output.
//
// Pipeline (one persistent CTA per SM, a contiguous range of (pair, 128-row
// tile) work items each, pairs that the inner solve left unchanged skipped):
//   * builder warps (7): load the FP64 rows of the tile, find each row's
//     exponent by warp shuffles, and write the digit tiles of Xh (A operand,
//     128 rows x 64 fp16, SWIZZLE_128B) into a ring of 6 shared-memory slots,
//     three digits per pass over the tile;
//   * one thread issues tcgen05.mma: B (the digits of D', built by the inner
//     solve, all s tiles resident per pair, brought in by one bulk copy) times
//     A_t for every u, with the tiles of u, u+1, ... adjacent so one product of
//     N = 64 run covers a run of diagonals; phase A forms the groups
//     d = 2..7 from A_1..A_6, phase B the groups d = 8..s+1 from A_1..A_s;
//   * epilogue warps (8: 4 TMEM lane quadrants x 2 column halves) drain each
//     group as soon as its last product is done (8 rotating TMEM slots of 64
//     columns), fold it into int64 Horner sums, park the phase-A sum in an
//     L2-resident scratch row, and write Y = X + corr.
// Wide pivots (more than 64 real-form positions: b > 32 columns per block in
// the complex case, b > 64 in the real one) are cut into 64-position tiles,
// T per pivot side: output tile nc of a 128-row tile is
//     Y_nc = X_nc + sum_kc X_kc (W2 - I)_(kc, nc),
// and each work item runs its T^2 tile products (kc, nc) through the same
// pipeline, each with its own row and column exponents. Their exact int128
// results are summed exactly (the smaller exponent's sum shifted to the
// larger one), one rounding to FP64 per output tile, and Y = X + corr is
// written once the item's last product is drained (in place: every tile of X
// is read by the products of every output tile).
//
// Every wait is bounded (tc::mbar_wait); a wait that runs out sets an error
// flag and every role leaves its loop, so the kernel returns with its TMEM
// freed.
#include "jj_common.cuh"
#include "jj_digits.cuh"
#include "jj_tc.cuh"

namespace jj {
namespace {

using namespace tc;

constexpr int UD_M = 128;                       // rows per tile (MMA M, TMEM lanes)
constexpr int UD_ASLOTS = 6;                    // A digit tiles in flight
constexpr int UD_TSLOTS = 8;                    // TMEM slots of 64 columns
constexpr int UD_EPI = 8;                       // epilogue warps 0..7
constexpr int UD_MMA = 8;                       // warp 8 issues the products
constexpr int UD_BLD0 = 9;                      // builder warps 9..15
constexpr int UD_BLD = 7;
constexpr int UD_THREADS = (UD_EPI + 1 + UD_BLD) * 32;
constexpr int UD_ATILE = UD_M * 128;            // 16 KB per A digit tile
constexpr int UD_PA = 6;                        // digits of phase A (groups 2..7)
constexpr int UD_RING = 4;                      // row-exponent ring (items)
constexpr int UD_TILE_LONGS = kUdPositions * UD_M;  // one 64-position tile of 64-bit words

// Per-CTA scratch (64-bit words): the parked phase-A sums; for wide pivots
// also the running int128 sums (lo, hi, exponent) of the current output tile
// and the FP64 corrections of every output tile.
__host__ __device__ constexpr size_t ud_scratch_longs(int tmax) {
    return (size_t)UD_TILE_LONGS +
           (tmax > 1 ? (size_t)UD_TILE_LONGS * 2 + UD_TILE_LONGS / 2 + (size_t)UD_TILE_LONGS * tmax : 0);
}

struct UdShared {
    unsigned long long a_full[UD_ASLOTS], a_empty[UD_ASLOTS];
    unsigned long long t_full[UD_TSLOTS], t_empty[UD_TSLOTS];
    unsigned long long r_full[UD_RING], r_empty[UD_RING];
    unsigned long long b_full, mma_done;
    int rexp[UD_RING][UD_M];
    uint32_t tmem_base;
    int abort;
    int q0, r0, count;
};

__device__ __forceinline__ int ud_tiles(const StepCtl &c, int q, int64_t m) {
    return (int)((pair_rows(c, q, m) + UD_M - 1) / UD_M);
}
__device__ __forceinline__ bool ud_active(const StepCtl &c, int q, int64_t m) {
    return !pair_passthrough(c, q) && ud_tiles(c, q, m) > 0;
}
// The work item after (q, r): the next tile of the pair, else the first tile
// of the next active pair.
__device__ __forceinline__ void ud_next(const StepCtl &c, int npairs, int64_t m, int &q, int &r) {
    if (++r < ud_tiles(c, q, m)) return;
    r = 0;
    do {
        ++q;
    } while (q < npairs && !ud_active(c, q, m));
}

__device__ __forceinline__ int64_t ud_gcol(const int32_t *pd, int c) {
    return c < pd[1] ? (int64_t)pd[0] + c : (int64_t)pd[2] + (c - pd[1]);
}

// 64-position tiles per side of a pivot with k columns (32 complex or 64 real
// columns per tile).
template <bool CPLX>
__host__ __device__ __forceinline__ int ud_ntiles(int k) {
    return CPLX ? (k + 31) / 32 : (k + 63) / 64;
}

// Arithmetic shift right of the two's-complement int128 (hi:lo) by n >= 0.
__device__ __forceinline__ void i128_sar(long long &hi, unsigned long long &lo, int n) {
    if (n <= 0) return;
    if (n >= 127) {
        lo = (unsigned long long)(hi >> 63);
        hi >>= 63;
    } else if (n >= 64) {
        lo = (unsigned long long)(hi >> (n - 64));
        hi >>= 63;
    } else {
        lo = (lo >> n) | ((unsigned long long)hi << (64 - n));
        hi >>= n;
    }
}

// Out of the normal range (never for the method's inputs): ldexp, kept out of
// line so that the common path carries none of its instructions.
__device__ __noinline__ double ud_scaled_slow(unsigned long long mant, int e, bool neg) {
    const double v = ldexp((double)mant, e);
    return neg ? -v : v;
}

// (hi:lo) as a two's-complement 128-bit integer times 2^e, rounded to the
// nearest double (ties to even): integer operations only.
__device__ __forceinline__ double i128_scaled_to_double(long long hi, unsigned long long lo, int e) {
    const unsigned long long sg = (unsigned long long)(hi >> 63);  // all ones when negative
    unsigned long long h = (unsigned long long)hi ^ sg, l = lo ^ sg;
    const unsigned long long l2 = l + (sg & 1ull);  // + 1 when negative
    h += (l2 < l) ? 1ull : 0ull;
    l = l2;
    if ((h | l) == 0ull) return 0.0;
    const int lz = h ? __clzll((long long)h) : 64 + __clzll((long long)l);  // 0..127
    unsigned long long top, rest;
    if (lz >= 64) {
        top = l << (lz - 64);
        rest = 0ull;
    } else if (lz == 0) {
        top = h;
        rest = l;
    } else {
        top = (h << lz) | (l >> (64 - lz));
        rest = l << lz;
    }
    unsigned long long mant = top >> 11;  // 53 bits, leading one at bit 52
    const unsigned long long rem = top & 0x7FFull;
    mant += (rem > 0x400ull || (rem == 0x400ull && (rest != 0ull || (mant & 1ull)))) ? 1ull : 0ull;
    int ex = 127 - lz + e;  // exponent of the leading bit
    if (mant >> 53) {
        mant >>= 1;
        ++ex;
    }
    const int biased = ex + 1023;
    if (__builtin_expect(biased < 1 || biased > 2046, 0)) return ud_scaled_slow(mant, ex - 52, sg != 0ull);
    return __longlong_as_double((long long)((sg << 63) | ((unsigned long long)biased << 52) |
                                            (mant & 0xFFFFFFFFFFFFFull)));
}

// WIDE: pivots of more than one 64-position tile per side (tmax > 1).
template <bool CPLX, bool WIDE>
__global__ void __launch_bounds__(UD_THREADS, 1) update_digits_kernel(
    const double *Gs, double *Gd, int64_t ld, int64_t m, const int32_t *__restrict__ pairs,
    int npairs, const int32_t *__restrict__ cexp, const uint8_t *__restrict__ wimg,
    const int32_t *__restrict__ wexp, int slices, int s, int tmax, long long *__restrict__ scratch,
    unsigned long long *__restrict__ counters, uint64_t wait_ns, StepCtl ctl) {
    extern __shared__ __align__(1024) uint8_t ud_smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>(((uintptr_t)ud_smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sB = sm;                                 // s tiles of 8 KB (digits of D')
    uint8_t *sA = sm + (size_t)s * kUpdSliceBytes;    // 6 slots of 16 KB (digits of Xh)
    __shared__ UdShared S;
    volatile int *abort_flag = &S.abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int hA = s < UD_PA ? s : UD_PA;  // digits (= groups) of phase A
    if (!WIDE) tmax = 1;
    const bool phaseB = s > UD_PA;

    // ---- set-up: barriers, TMEM, this CTA's range of work items ----
    if (warp == UD_MMA) {
        tmem_alloc(su32(&S.tmem_base), 512);
        if (lane == 0) {
            for (int i = 0; i < UD_ASLOTS; ++i) {
                mbar_init(su32(&S.a_full[i]), UD_BLD);
                mbar_init(su32(&S.a_empty[i]), 1);
            }
            for (int i = 0; i < UD_TSLOTS; ++i) {
                mbar_init(su32(&S.t_full[i]), 1);
                mbar_init(su32(&S.t_empty[i]), UD_EPI);
            }
            for (int i = 0; i < UD_RING; ++i) {
                mbar_init(su32(&S.r_full[i]), UD_BLD);
                mbar_init(su32(&S.r_empty[i]), UD_EPI);
            }
            mbar_init(su32(&S.b_full), 1);
            mbar_init(su32(&S.mma_done), 1);
            mbar_init_fence();
            S.abort = 0;
        }
        // active tiles of all pairs, and the first item of this CTA's share
        long long total = 0;
        for (int base = 0; base < npairs; base += 32) {
            const int q = base + lane;
            int t = (q < npairs && ud_active(ctl, q, m)) ? ud_tiles(ctl, q, m) : 0;
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
            const int t = (q < npairs && ud_active(ctl, q, m)) ? ud_tiles(ctl, q, m) : 0;
            int inc = t;  // inclusive prefix over the lanes
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

    if (warp < UD_EPI) {
        // ------------------------------------------------------------------
        // Epilogue: thread = output row (TMEM lane), 32 output positions.
        // ------------------------------------------------------------------
        const int quad = warp & 3, hh = warp >> 2;
        const int rl = quad * 32 + lane;
        long long *scr = scratch + (size_t)blockIdx.x * ud_scratch_longs(tmax);
        unsigned long long *slo = reinterpret_cast<unsigned long long *>(scr + UD_TILE_LONGS);
        long long *shi = scr + 2 * UD_TILE_LONGS;
        int *sex = reinterpret_cast<int *>(scr + 3 * UD_TILE_LONGS);
        double *ysum = reinterpret_cast<double *>(scr + 3 * UD_TILE_LONGS + UD_TILE_LONGS / 2);
        int q = S.q0, r = S.r0;
        long long acc[32];
        // Drain n = 1 or 2 consecutive groups g (and g + 1) into the Horner sums
        // (int64, base 256; |S_d| < 11 * 2^20); both TMEM slots are released
        // after the pair. False when a wait ran out.
        auto drain = [&](long long g, int n, bool first) -> bool {
            for (int i = 0; i < n; ++i) {
                const int slot = (int)((g + i) & (UD_TSLOTS - 1));
                const uint32_t par = (uint32_t)(((g + i) >> 3) & 1);
                const bool ok = __all_sync(0xffffffffu,
                                           !*abort_flag && mbar_wait(su32(&S.t_full[slot]), par, wait_ns));
                if (!ok) {
                    *abort_flag = 1;
                    return false;
                }
            }
            tc_fence_after();
            const int s0 = (int)(g & (UD_TSLOTS - 1)), s1 = (int)((g + 1) & (UD_TSLOTS - 1));
            const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(hh * 32);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                uint32_t v0[8], v1[8];
                tmem_ld8(lane_base + (uint32_t)(s0 * 64 + h * 8), v0);
                if (n == 2) tmem_ld8(lane_base + (uint32_t)(s1 * 64 + h * 8), v1);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int i0 = __float2int_rn(__uint_as_float(v0[c]));  // exact integers
                    long long& a = acc[h * 8 + c];
                    if (n == 2) {
                        const long long pr = (long long)i0 * 256 + __float2int_rn(__uint_as_float(v1[c]));
                        a = first ? pr : a * 65536 + pr;
                    } else {
                        a = first ? (long long)i0 : a * 256 + i0;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(su32(&S.t_empty[s0]));
                if (n == 2) mbar_arrive(su32(&S.t_empty[s1]));
            }
            return true;
        };
        // groups [d_lo, d_hi] of item j, in pairs
        auto drain_range = [&](long long g0, int d_lo, int d_hi) -> bool {
            for (int d = d_lo; d <= d_hi; d += 2)
                if (!drain(g0 + d - 2, d + 1 <= d_hi ? 2 : 1, d == d_lo)) return false;
            return true;
        };
        int J = 0;  // tile products of this CTA so far
        for (int j = 0; j < count; ++j) {
            if (*abort_flag) break;
            const int32_t *pd = pairs + 4 * q;
            const int k = pd[1] + pd[3];
            const int Tq = WIDE ? ud_ntiles<CPLX>(k) : 1;
            const int64_t rows = pair_rows(ctl, q, m);
            const int64_t l = (int64_t)r * UD_M + rl;
            bool ok = true;
            for (int sp = 0; sp < Tq * Tq; ++sp, ++J) {
                const int nc = sp / Tq, kc = sp % Tq;
                const long long g0 = (long long)J * s;
                ok = drain_range(g0, 2, hA + 1);
                if (!ok) break;
                if (phaseB) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) scr[(size_t)(hh * 32 + c) * UD_M + rl] = acc[c];
                    ok = drain_range(g0, UD_PA + 2, s + 1);
                    if (!ok) break;
                }
                const int rho = (int)(J % UD_RING);
                if (!__all_sync(0xffffffffu,
                                mbar_wait(su32(&S.r_full[rho]), (uint32_t)((J / UD_RING) & 1), wait_ns))) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                const int re = S.rexp[rho][rl];
                const int32_t *wx = wexp + ((size_t)q * tmax * tmax + nc * tmax + kc) * kUdPositions + hh * 32;
                // pivot column of output position hh * 32 + cc of tile nc
                auto pcol = [&](int cc) { return CPLX ? 32 * nc + cc : 64 * nc + hh * 32 + cc; };
                if (l < rows && (!WIDE || Tq == 1)) {
                    // Y = X + corr, 4 outputs at a time: all loads of a batch are
                    // issued before its stores (Gd may be Gs, so a load cannot move
                    // above a store)
#pragma unroll
                    for (int cb = 0; cb < 32; cb += 4) {
                        int64_t idx[4];
                        double xv[4];
                        long long av[4];
                        int wv[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int cc = pcol(cb + c);
                            idx[c] = cc < k ? (CPLX ? (ud_gcol(pd, cc) * ld + l) * 2 + hh : ud_gcol(pd, cc) * ld + l)
                                            : -1;
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            xv[c] = idx[c] >= 0 ? Gs[idx[c]] : 0.0;
                            av[c] = phaseB ? scr[(size_t)(hh * 32 + cb + c) * UD_M + rl] : 0ll;
                            wv[c] = wx[cb + c];
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            if (idx[c] < 0) continue;
                            long long hi;
                            unsigned long long lo;
                            const long long b = acc[cb + c];
                            if (phaseB) {
                                // T = accA 2^(8 (s - 6)) + accB
                                const int sh = 8 * (s - UD_PA);
                                const unsigned long long al = (unsigned long long)av[c] << sh;
                                const long long ah = av[c] >> (64 - sh);
                                lo = al + (unsigned long long)b;
                                hi = ah + (b >> 63) + (lo < al ? 1 : 0);
                            } else {
                                lo = (unsigned long long)b;
                                hi = b >> 63;
                            }
                            Gd[idx[c]] = xv[c] + i128_scaled_to_double(hi, lo, re + wv[c] + 4 - 8 * (s + 1));
                        }
                    }
                } else if (WIDE && l < rows) {
                    // wide pivot: add this tile product to the running int128 sum
                    // of output tile nc; its last one is rounded to FP64
#pragma unroll 4
                    for (int c = 0; c < 32; ++c) {
                        if (pcol(c) >= k) continue;
                        long long hi;
                        unsigned long long lo;
                        const long long b = acc[c];
                        const size_t si = (size_t)(hh * 32 + c) * UD_M + rl;
                        if (phaseB) {
                            const long long a = scr[si];
                            const int sh = 8 * (s - UD_PA);
                            const unsigned long long al = (unsigned long long)a << sh;
                            const long long ah = a >> (64 - sh);
                            lo = al + (unsigned long long)b;
                            hi = ah + (b >> 63) + (lo < al ? 1 : 0);
                        } else {
                            lo = (unsigned long long)b;
                            hi = b >> 63;
                        }
                        int e = re + wx[c];
                        if (kc > 0) {
                            unsigned long long rlo = slo[si];
                            long long rhi = shi[si];
                            const int re2 = sex[si];
                            if (e > re2) {
                                i128_sar(rhi, rlo, e - re2);
                            } else {
                                i128_sar(hi, lo, re2 - e);
                                e = re2;
                            }
                            const unsigned long long sl = rlo + lo;
                            hi = rhi + hi + (sl < rlo ? 1 : 0);
                            lo = sl;
                        }
                        if (kc == Tq - 1) {
                            ysum[(size_t)(nc * kUdPositions + hh * 32 + c) * UD_M + rl] =
                                i128_scaled_to_double(hi, lo, e + 4 - 8 * (s + 1));
                        } else {
                            slo[si] = lo;
                            shi[si] = hi;
                            sex[si] = e;
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(su32(&S.r_empty[rho]));
            }
            if (!ok) break;
            if (WIDE && Tq > 1 && l < rows) {
                // the item's products are all drained, so every tile of X has
                // been read: Y = X + corr for every output tile
                for (int nc = 0; nc < Tq; ++nc) {
#pragma unroll
                    for (int cb = 0; cb < 32; cb += 4) {
                        int64_t idx[4];
                        double xv[4], yv[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int cc = CPLX ? 32 * nc + cb + c : 64 * nc + hh * 32 + cb + c;
                            idx[c] = cc < k ? (CPLX ? (ud_gcol(pd, cc) * ld + l) * 2 + hh : ud_gcol(pd, cc) * ld + l)
                                            : -1;
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            xv[c] = idx[c] >= 0 ? Gs[idx[c]] : 0.0;
                            yv[c] = idx[c] >= 0 ? ysum[(size_t)(nc * kUdPositions + hh * 32 + cb + c) * UD_M + rl] : 0.0;
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (idx[c] >= 0) Gd[idx[c]] = xv[c] + yv[c];
                    }
                }
            }
            ud_next(ctl, npairs, m, q, r);
        }
    } else if (warp == UD_MMA) {
        // ------------------------------------------------------------------
        // Product issue (one thread).
        // ------------------------------------------------------------------
        if (lane == 0) {
            int q = S.q0, r = S.r0;
            long long prev_key = -1;
            uint32_t bpar = 0, dpar = 0;
            // a bulk copy / a commit whose completion has not been seen yet (a
            // barrier must not complete two phases unobserved: its parity wait
            // could not tell them apart)
            bool b_pending = false, d_pending = false;
            const uint32_t a_base = su32(sA), b_base = su32(sB);
            bool ok = true;
            auto waitb = [&](unsigned long long *bar, uint32_t par) {
                if (ok && (*abort_flag || !mbar_wait(su32(bar), par, wait_ns))) {
                    ok = false;
                    *abort_flag = 1;
                }
            };
            // products A_t x B_u for u in [u_lo, u_hi] into the groups t + u of item j
            auto issue = [&](long long g0, int t, int u_lo, int u_hi) {
                const uint32_t a0 = a_base + (uint32_t)(((t - 1) % UD_ASLOTS) * UD_ATILE);
                for (int u = u_lo; u <= u_hi;) {
                    const long long g = g0 + t + u - 2;
                    const int slot = (int)(g & (UD_TSLOTS - 1));
                    int run = u_hi - u + 1;
                    run = min(run, 4);
                    run = min(run, UD_TSLOTS - slot);
                    const uint32_t id = idesc_f16(UD_M, 64 * run);
                    const uint32_t b0 = b_base + (uint32_t)((u - 1) * kUpdSliceBytes);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        mma_f16(tmem + (uint32_t)(slot * 64), desc_sw128(a0 + ks * 32),
                                desc_sw128(b0 + ks * 32), id, (t == 1 && ks == 0) ? 0u : 1u);
                    u += run;
                }
            };
            // before the first product of groups [d_lo, d_hi] of item j: their
            // TMEM slots have been drained by the epilogue
            auto wait_slots = [&](long long g0, int d_lo, int d_hi) {
                for (int d = d_lo; d <= d_hi; ++d) {
                    const long long g = g0 + d - 2;
                    if (g >= UD_TSLOTS) waitb(&S.t_empty[g & (UD_TSLOTS - 1)], (uint32_t)(((g >> 3) - 1) & 1));
                }
            };
            int J = 0;  // tile products of this CTA so far
            for (int j = 0; j < count && ok; ++j) {
                const int Tq = WIDE ? ud_ntiles<CPLX>(pairs[4 * q + 1] + pairs[4 * q + 3]) : 1;
                for (int sp = 0; sp < Tq * Tq && ok; ++sp, ++J) {
                    const int nc = sp / Tq, kc = sp % Tq;
                    const long long key = ((long long)q * tmax + nc) * tmax + kc;  // W tile (q, kc, nc)
                    if (key != prev_key) {
                        // the B tiles of the new W tile, once the products reading the old ones are done
                        if (prev_key >= 0) {
                            mma_commit(su32(&S.mma_done));
                            d_pending = true;
                            waitb(&S.mma_done, dpar);
                            if (!ok) break;
                            d_pending = false;
                            dpar ^= 1u;
                        }
                        mbar_expect_tx(su32(&S.b_full), (uint32_t)(s * kUpdSliceBytes));
                        bulk_g2s(b_base, wimg + (size_t)key * slices * kUpdSliceBytes,
                                 (uint32_t)(s * kUpdSliceBytes), su32(&S.b_full));
                        b_pending = true;
                        waitb(&S.b_full, bpar);
                        if (!ok) break;
                        b_pending = false;
                        bpar ^= 1u;
                        prev_key = key;
                    }
                    const long long g0 = (long long)J * s;
                    // phase A: groups 2..hA+1 from A_1..A_hA
                    for (int t = 1; t <= hA && ok; ++t) {
                        const int sl = t - 1;
                        const int nuse = (sl + UD_PA + 1 <= s) ? 2 : 1;
                        waitb(&S.a_full[sl], (uint32_t)((J * nuse) & 1));
                        if (t == 1) wait_slots(g0, 2, hA + 1);
                        if (!ok) break;
                        tc_fence_after();
                        issue(g0, t, 1, hA + 1 - t);
                        const long long gf = g0 + t - 1;  // group t + 1 is complete
                        mma_commit(su32(&S.t_full[gf & (UD_TSLOTS - 1)]));
                        if (!phaseB) mma_commit(su32(&S.a_empty[sl]));
                    }
                    // phase B: groups 8..s+1 from A_1..A_s
                    for (int t = 1; phaseB && t <= s && ok; ++t) {
                        const int sl = (t - 1) % UD_ASLOTS;
                        if (t > UD_PA) waitb(&S.a_full[sl], (uint32_t)((J * 2 + 1) & 1));
                        if (t == 1) wait_slots(g0, UD_PA + 2, s + 1);
                        if (!ok) break;
                        tc_fence_after();
                        issue(g0, t, max(1, UD_PA + 2 - t), s + 1 - t);
                        mma_commit(su32(&S.a_empty[sl]));
                        if (t + 1 >= UD_PA + 2) mma_commit(su32(&S.t_full[(g0 + t - 1) & (UD_TSLOTS - 1)]));
                    }
                }
                ud_next(ctl, npairs, m, q, r);
            }
            // Every product and copy has completed before the TMEM and the shared
            // memory are released; after a wait ran out these waits keep the
            // default bound (the operations in flight still finish quickly).
            if (!d_pending) mma_commit(su32(&S.mma_done));
            if (!mbar_wait(su32(&S.mma_done), dpar, kWaitLimitNs)) *abort_flag = 1;
            if (b_pending && !mbar_wait(su32(&S.b_full), bpar, kWaitLimitNs)) *abort_flag = 1;
        }
    } else {
        // ------------------------------------------------------------------
        // Builders: digits of Xh = X D^-1 relative to each row's exponent.
        // A pass writes three digits (one 24-bit window of each value's 88-bit
        // biased image) of the warp's rows of the tile, in two batches of
        // tasks; each batch issues all its loads at once (the first batch before
        // the wait for free slots, so that the loads' latency overlaps it). The
        // row exponents are found in the first pass and kept in shared memory.
        // Each lane stores its u32 items in an order rotated by its row, so that
        // the 32 lanes of one store instruction hit 32 different banks of the
        // swizzled tile.
        // ------------------------------------------------------------------
        const int bw = warp - UD_BLD0;
        int q = S.q0, r = S.r0;
        bool ok = true;
        auto waitb = [&](unsigned long long *bar, uint32_t par) {
            if (!ok) return;
            if (!__all_sync(0xffffffffu, !*abort_flag && mbar_wait(su32(bar), par, wait_ns))) {
                ok = false;
                *abort_flag = 1;
            }
        };
        // complex: a task is 2 rows x 32 columns (lane: column pair 2c', 2c'+1 of
        // row rr); real: 4 rows x 64 columns (lane: columns 8c'..8c'+7 of row rr)
        constexpr int NV = CPLX ? 4 : 8;          // values per lane and task
        constexpr int NI = NV / 2;                // u32 items (two positions) per lane and task
        constexpr int TASKS = CPLX ? 64 : 32;     // tasks per tile
        constexpr int RPT = CPLX ? 2 : 4;         // rows per task
        constexpr int TPW = (TASKS + UD_BLD - 1) / UD_BLD;  // tasks per builder warp (at most)
        constexpr int HB = (TPW + 1) / 2;         // tasks per batch
        constexpr int NC = CPLX ? 2 : NV;         // columns per lane
        const int cl = CPLX ? (lane & 15) : (lane & 7);
        const int rr = CPLX ? (lane >> 4) : (lane >> 3);
        // value v of this lane sits at real-form position vpos[v]; item i is the
        // value pair (2i, 2i + 1). Complex: [re c0, re c1, im c0, im c1], with the
        // two items swapped for rr = 1; real: columns 8c' + ((v + 2 rr) mod 8).
        int vcol[NV];  // pivot column of value v
        int ipos[NI];  // position of item i's first value
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (CPLX) {
                vcol[v] = 2 * cl + (v & 1);
            } else {
                vcol[v] = 8 * cl + ((v + 2 * rr) & 7);
            }
        }
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            if (CPLX)
                ipos[i] = ((i ^ rr) == 0) ? 2 * cl : 32 + 2 * cl;
            else
                ipos[i] = vcol[2 * i];
        }
        uint32_t ichunk[NI], ilow[NI];  // 16-byte chunk and byte of item i within a row
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            ichunk[i] = (uint32_t)(ipos[i] * 2) >> 4;
            ilow[i] = (uint32_t)(ipos[i] * 2) & 15u;
        }
        int J = 0;  // tile products of this CTA so far
        for (int j = 0; j < count && ok; ++j) {
            const int32_t *pd = pairs + 4 * q;
            const int k = pd[1] + pd[3];
            const int Tq = WIDE ? ud_ntiles<CPLX>(k) : 1;
            const int64_t rows = pair_rows(ctl, q, m);
            const int64_t l0 = (int64_t)r * UD_M;
            for (int sp = 0; sp < Tq * Tq && ok; ++sp, ++J) {
                const int kc = sp % Tq;  // the tile of X this product reads
                const int rho = (int)(J % UD_RING);
                int64_t colx[NC];
                int ex[NV];
#pragma unroll
                for (int v = 0; v < NC; ++v) {
                    const int c = CPLX ? 32 * kc + 2 * cl + v : 64 * kc + vcol[v];
                    colx[v] = c < k ? ud_gcol(pd, c) : -1;
                }
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int64_t cx = colx[CPLX ? (v & 1) : v];
                    ex[v] = cx >= 0 ? cexp[cx] : -1021;
                }
                if (J >= UD_RING) waitb(&S.r_empty[rho], (uint32_t)((J / UD_RING - 1) & 1));
                for (int p = 0; p < 4 && ok; ++p) {
                    const int t0 = 3 * p + 1;
                    if (t0 > s) break;
                    const int t1 = min(3 * p + 3, s);
                    for (int hb = 0; hb < 2 && ok; ++hb) {
                        // this batch's values, all loads in flight together
                        double x[HB][NV];
#pragma unroll
                        for (int i = 0; i < HB; ++i) {
                            const int task = bw + UD_BLD * (hb * HB + i);
                            const bool has = hb * HB + i < TPW && task < TASKS;
                            const int64_t l = l0 + task * RPT + rr;
#pragma unroll
                            for (int v = 0; v < NC; ++v) {
                                const bool in = has && colx[v] >= 0 && l < rows;
                                if (CPLX) {
                                    double2 z = make_double2(0.0, 0.0);
                                    if (in) z = reinterpret_cast<const double2 *>(Gs)[colx[v] * ld + l];
                                    x[i][v] = rr ? z.y : z.x;      // first item: re (rr = 0) or im
                                    x[i][v + 2] = rr ? z.x : z.y;
                                } else {
                                    x[i][v] = in ? Gs[colx[v] * ld + l] : 0.0;
                                }
                            }
                        }
                        if (hb == 0) {  // the slots of this pass's digits are free
                            for (int t = t0; t <= t1; ++t) {
                                const int sl = (t - 1) % UD_ASLOTS;
                                const int nuse = (sl + UD_PA + 1 <= s) ? 2 : 1;
                                const long long use = (long long)J * nuse + (t > UD_PA ? 1 : 0);
                                if (use >= 1) waitb(&S.a_empty[sl], (uint32_t)((use - 1) & 1));
                            }
                            if (!ok) break;
                        }
                        uint8_t *slotp[3];  // slots of the pass's digits t0, t0 + 1, t0 + 2
#pragma unroll
                        for (int dd = 0; dd < 3; ++dd)
                            slotp[dd] = sA + (size_t)((t0 - 1 + dd) % UD_ASLOTS) * UD_ATILE;
#pragma unroll
                        for (int i = 0; i < HB; ++i) {
                            const int task = bw + UD_BLD * (hb * HB + i);
                            if (hb * HB + i >= TPW || task >= TASKS) break;
                            const int row = task * RPT + rr;  // row of the tile
                            int rexp;
                            if (p == 0) {
                                // row exponent: max over the row of exp(x) - e_a
                                int mx = -100000;
#pragma unroll
                                for (int v = 0; v < NV; ++v) {
                                    const unsigned long long mb = dg_mag_bits(x[i][v]);
                                    if (mb) mx = max(mx, dg_exp_of_bits(mb) - ex[v]);
                                }
#pragma unroll
                                for (int o = 1; o < (CPLX ? 16 : 8); o <<= 1)
                                    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                                rexp = mx == -100000 ? -1021 : mx;
                                if (cl == 0) S.rexp[rho][row] = rexp;
                            } else {
                                rexp = S.rexp[rho][row];
                            }
                            // complex: the value order differs between rr = 0 and 1, and
                            // e_a is the same for the real and imaginary part of a column
                            uint32_t w[NV];
#pragma unroll
                            for (int v = 0; v < NV; ++v) w[v] = dg_window24(x[i][v], rexp + ex[v], p);
                            const uint32_t rowbase = (uint32_t)row * 128u, x7 = (uint32_t)row & 7u;
#pragma unroll
                            for (int it = 0; it < NI; ++it) {
                                const uint32_t off = rowbase + ((ichunk[it] ^ x7) << 4) + ilow[it];
#pragma unroll
                                for (int dd = 0; dd < 3; ++dd) {
                                    if (t0 + dd > t1) break;
                                    const uint32_t u0 = (w[2 * it] >> (16 - 8 * dd)) & 255u;
                                    const uint32_t u1 = (w[2 * it + 1] >> (16 - 8 * dd)) & 255u;
                                    *reinterpret_cast<uint32_t *>(slotp[dd] + off) = dg_pack2(u0, u1);
                                }
                            }
                        }
                    }
                    if (!ok) break;
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        for (int t = t0; t <= t1; ++t) mbar_arrive(su32(&S.a_full[(t - 1) % UD_ASLOTS]));
                        if (p == 0) mbar_arrive(su32(&S.r_full[rho]));
                    }
                }
            }
            ud_next(ctl, npairs, m, q, r);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && S.abort && counters) atomicOr(&counters[kCntErr], kErrTimeout);
    if (warp == UD_MMA) tmem_dealloc(tmem, 512);
}

// The W-side operand of the update (ud_wimage_build) for every active pair of
// a step, from W_P in global memory: one block per (pair, W tile (kc, nc)),
// images at [pair][nc][kc] with tmax tiles per side. The solver's inner solve
// builds the image of a narrow pivot itself; this kernel serves wide pivots
// and the building-block entry point.
template <bool CPLX>
__global__ void __launch_bounds__(256) wimage_kernel(const double *__restrict__ W, int kmax,
                                                     const int32_t *__restrict__ pairs,
                                                     const int32_t *__restrict__ cexp, int slices,
                                                     int tmax, uint8_t *__restrict__ img,
                                                     int32_t *__restrict__ wexp, StepCtl ctl) {
    constexpr int E = CPLX ? 2 : 1;
    constexpr int CW = CPLX ? 32 : 64;  // pivot columns per tile
    __shared__ int s_xexp[kUdPositions], s_wexp[kUdPositions];
    const int q = blockIdx.x, sp = blockIdx.y;
    if (pair_passthrough(ctl, q)) return;
    const int32_t *pd = pairs + 4 * q;
    const int k = pd[1] + pd[3];
    const int Tq = ud_ntiles<CPLX>(k);
    const int nc = sp / tmax, kc = sp % tmax;
    if (nc >= Tq || kc >= Tq) return;
    const int kr = min(CW, k - CW * kc), kn = min(CW, k - CW * nc);
    for (int a = threadIdx.x; a < kUdPositions; a += blockDim.x) {
        const int c = CPLX ? (a & 31) : a;
        s_xexp[a] = c < kr ? cexp[ud_gcol(pd, CW * kc + c)] : -1021;
    }
    __syncthreads();
    const double *Wp = W + (size_t)q * kmax * kmax * E;
    auto wacc = [&](int rr, int cc, int part) -> double {
        return Wp[((size_t)(CW * nc + cc) * kmax + CW * kc + rr) * E + part];
    };
    const size_t tile = (size_t)q * tmax * tmax + sp;
    ud_wimage_build<CPLX>(wacc, kr, kn, kc == nc, s_xexp, s_wexp, slices,
                          img + tile * slices * kUpdSliceBytes, wexp + tile * kUdPositions, threadIdx.x,
                          blockDim.x);
}

}  // namespace

int ud_max_tiles(bool cplx, int kmax) { return cplx ? ud_ntiles<true>(kmax) : ud_ntiles<false>(kmax); }

size_t ud_scratch_bytes(int nctas, int tmax) {
    return (size_t)nctas * ud_scratch_longs(tmax) * sizeof(long long);
}

int ud_num_ctas() {
    static int sms[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!sms[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        sms[dev] = v;
    }
    return sms[dev];
}

cudaError_t launch_wimage(bool cplx, const double *W, int kmax, const int32_t *pairs, int npairs,
                          const int32_t *cexp, const UpdDigits &ud, cudaStream_t st, StepCtl ctl) {
    if (npairs <= 0) return cudaSuccess;
    const int tmax = ud_max_tiles(cplx, kmax);
    if (tmax > kUdMaxTiles || ud.slices < 1 || ud.slices > kUdMaxSlices) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)npairs, (unsigned)(tmax * tmax));
    if (cplx)
        wimage_kernel<true><<<grid, 256, 0, st>>>(W, kmax, pairs, cexp, ud.slices, tmax, ud.img, ud.wexp, ctl);
    else
        wimage_kernel<false><<<grid, 256, 0, st>>>(W, kmax, pairs, cexp, ud.slices, tmax, ud.img, ud.wexp, ctl);
    return cudaGetLastError();
}

cudaError_t launch_update_digits(bool cplx, const double *Gs, double *Gd, int64_t ld, int64_t m,
                                 int64_t ncols, const int32_t *pairs, int npairs, int kmax, int maxblk,
                                 const int32_t *cexp, const UpdDigits &ud, long long *scratch, int nctas,
                                 unsigned long long *counters, cudaStream_t st, StepCtl ctl) {
    if (npairs <= 0) return cudaSuccess;
    if (Gd != Gs && ctl.flags) return cudaErrorInvalidValue;
    if (maxblk > 0 && ud.slices == kUdMaxSlices && un_supported(cplx, Gs, ld, m, ncols, kmax, maxblk))
        return launch_update_narrow(cplx, Gs, Gd, ld, m, ncols, pairs, npairs, cexp, ud, nctas, counters, st, ctl);
    const int s = ud.slices;
    const int tmax = ud_max_tiles(cplx, kmax);
    if (tmax > kUdMaxTiles || s < 1 || s > kUdMaxSlices || !ud.img || !ud.wexp || !scratch || nctas < 1)
        return cudaErrorInvalidValue;
    // skipped pairs are left in place, so an out-of-place update needs every pair active
    if (Gd != Gs && ctl.flags) return cudaErrorInvalidValue;
    const size_t smem = (size_t)s * kUpdSliceBytes + (size_t)UD_ASLOTS * UD_ATILE + 1024;
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<nctas, UD_THREADS, smem, st>>>(Gs, Gd, ld, m, pairs, npairs, cexp, ud.img, ud.wexp, ud.slices, s,
                                              tmax, scratch, counters, ctl.wait_ns, ctl);
        return cudaSuccess;
    };
    cudaError_t e;
    if (cplx)
        e = tmax > 1 ? run(update_digits_kernel<true, true>) : run(update_digits_kernel<true, false>);
    else
        e = tmax > 1 ? run(update_digits_kernel<false, true>) : run(update_digits_kernel<false, false>);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace jj
