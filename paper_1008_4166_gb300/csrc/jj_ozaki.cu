// Split-precision (Ozaki scheme I) Gram and update on the tcgen05 tensor cores.
//
// Both dense contractions of the blocked method -- the pivot Gram
// A_P = [G_i G_j]^* [G_i G_j] (3.6) and the update [G_i G_j] W_P (2.9) -- run as
// sums of exact fp16 x fp16 -> fp32 products on the tensor cores:
//
//   * Real form. A complex pivot X = Xr + i Xi (m x k) is handled as the real
//     m x 2k matrix [Xr Xi]; its Gram C = [Xr Xi]^T [Xr Xi] gives
//     Re A = C11 + C22, Im A = C12 - C21, and the update is
//     [Yr Yi] = [Xr Xi] [[Wr, Wi], [-Wi, Wr]].
//   * Splitting (error-free slicing of Ozaki, Ogita, Oishi and Rump, 2012, in
//     the fixed-point form used for tensor cores by Mukunoki, Ozaki, Ogita and
//     Imamura, 2020): every FP64 entry x of a vector with common exponent e
//     (all |x| < 2^e) is written as x = 2^e sum_{t=1..s} 2^{-7t} d_t + r with
//     integer digits |d_t| <= 127 and 0 <= |r| < 2^{e - 7s}. The digits are
//     taken from the bits of x with integer shifts only (no FP64 arithmetic)
//     and stored as fp16, which holds them exactly.
//   * Products of digit matrices A_t^T B_u are exact integers; all products of
//     one diagonal d = t + u (same weight 2^{-7d}) accumulate in one fp32 TMEM
//     accumulator, exactly, as long as (#products) * K * 127^2 < 2^24.
//   * Each diagonal's fp32 sum is converted to an integer and added, shifted
//     by its weight, into integer fixed-point accumulators: int128 for the Gram
//     (every product kept exactly; the Gram must resolve off-diagonals far
//     below its largest entries), int64 for the update. One FP64 conversion
//     and one scaling per output entry end the computation.
//
// Shared-memory operands use the canonical K-major SWIZZLE_128B layout:
// 128-byte rows (64 fp16 along K), 8-row groups 1024 bytes apart, the 16-byte
// chunks of row r XOR-ed with r mod 8. They are written by the producer
// threads (the digits are computed, not copied), then fenced to the async
// proxy before the single issuing thread launches tcgen05.mma.
#include <cstring>

#include "jj_common.cuh"
#include "jj_tc.cuh"

namespace jj {

constexpr int kBeta = 7;          // bits per digit
constexpr int kOzMaxK2 = 256;     // real width 2k (complex) or k (real) handled here

namespace {

using namespace tc;

// ---------------------------------------------------------------------------
// Digits
// ---------------------------------------------------------------------------
// Sign and magnitude tests on the bit pattern of a double: on this part an FP64
// comparison or absolute value runs on the FP64 pipe, 64 times slower than the
// integer ALU, so the digit kernels never touch FP64 arithmetic.
__device__ __forceinline__ bool neg_bits(double x) { return __double_as_longlong(x) < 0; }
__device__ __forceinline__ unsigned long long mag_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// Exponent e with |x| < 2^e for the magnitude bit pattern `mag` (a non-negative
// double's bits); zero and subnormals give the smallest normal exponent.
__device__ __forceinline__ int exp_of_bits(unsigned long long mag) {
    const int E = (int)((mag >> 52) & 0x7FF);
    return E == 0 ? -1021 : E - 1022;
}

// q = floor(|x| 2^(63-e)) for |x| < 2^e, by shifting the 53-bit significand.
__device__ __forceinline__ unsigned long long fixed63(double x, int e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0) return 0ull;  // zero / subnormal: below every digit kept here
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - 1012 - e;  // <= 10 because |x| < 2^e
    if (sh >= 0) return mant << sh;
    if (sh <= -64) return 0ull;
    return mant >> (-sh);
}

// ---------------------------------------------------------------------------
// Column exponents of the work matrix: e_c with max_l max(|Re|, |Im|) < 2^e_c.
// ---------------------------------------------------------------------------
template <bool CPLX>
__global__ void __launch_bounds__(256) colexp_kernel(const double *__restrict__ G, int64_t ld,
                                                      int64_t m, int32_t *__restrict__ cexp) {
    __shared__ unsigned long long sh[8];
    const int64_t c = blockIdx.x;
    unsigned long long mx = 0;
    const double *g = G + c * ld * (CPLX ? 2 : 1);
    const int64_t cnt = m * (CPLX ? 2 : 1);
    for (int64_t i = threadIdx.x; i < cnt; i += 256) {
        const unsigned long long v = mag_bits(g[i]);
        mx = v > mx ? v : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) mx = sh[w] > mx ? sh[w] : mx;
        cexp[c] = exp_of_bits(mx);
    }
}

// Column exponents of the pivot columns of the pairs of one step, over the
// rows of each pair's problem: one block per (pivot column, pair). Pairs the
// Gram will skip (unchanged since found diagonal) are left out.
template <bool CPLX>
__global__ void __launch_bounds__(256) colexp_pairs_kernel(const double *__restrict__ G, int64_t ld,
                                                            int64_t m, const int32_t *__restrict__ pairs,
                                                            int32_t *__restrict__ cexp, StepCtl ctl) {
    __shared__ unsigned long long sh[8];
    const int q = blockIdx.y;
    const int32_t *pd = pairs + 4 * q;
    const int a = blockIdx.x;
    if (a >= pd[1] + pd[3]) return;
    if (ctl.mod_step && pair_skip_decide(ctl, pd, q)) return;
    const int64_t c = a < pd[1] ? (int64_t)pd[0] + a : (int64_t)pd[2] + (a - pd[1]);
    unsigned long long mx = 0;
    const double *g = G + c * ld * (CPLX ? 2 : 1);
    const int64_t cnt = pair_rows(ctl, q, m) * (CPLX ? 2 : 1);
    for (int64_t i = threadIdx.x; i < cnt; i += 256) {
        const unsigned long long v = mag_bits(g[i]);
        mx = v > mx ? v : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) mx = sh[w] > mx ? sh[w] : mx;
        cexp[c] = exp_of_bits(mx);
    }
}

// ---------------------------------------------------------------------------
// Gram: one block per (row range, pair). The pivot's K2 real columns are the
// 64 rows of the A operand (M = 64) and, the Gram being X^T X, the same
// shared-memory tile serves as the B operand. With s = 8 digits (56 bits;
// the Gram error stays below sqrt(m) 2^-56 of ||x_a|| ||x_b|| by the
// Cauchy-Schwarz inequality), the products of one diagonal d = t + u
// (d - 1 <= 8 of them) form one TMEM group, and the 8 groups occupy the 512
// TMEM columns at once. Rows of G arrive 64 at a time in two shared-memory
// buffers (digits of the next 64 rows are built while the tensor cores read
// the current ones); every group accumulates 128 rows in TMEM, which keeps its
// fp32 sum an exact integer below 2^24 (8 * 128 * 127^2 < 2^24), and is then
// drained into two signed 64-bit words per output (no carries until the end).
// At the end each block adds its partial sums atomically into the global
// int128 accumulator (lo, hi words with an explicit carry).
//
// Wide pivots (K2 > 64) are cut into 64-position tiles; the grid's third
// dimension runs over the tile pairs (ta, tb), ta <= tb, of the upper
// triangle (the Gram is symmetric and its integer sums are exact, so the lower
// tiles are the transposes). A diagonal tile is the case above; an
// off-diagonal one takes its two operands from two buffers, one stage deep.
// ---------------------------------------------------------------------------
constexpr int GZ_THREADS = 512;
constexpr int GZ_KC = 64;                 // rows of G per shared-memory buffer
constexpr int GZ_SLICE_BYTES = 64 * 128;  // 64 operand rows x 128 bytes
constexpr int GZ_SLICES = 8;              // digits of the Gram operands
constexpr int GZ_BUF_BYTES = GZ_SLICES * GZ_SLICE_BYTES;

constexpr int GZ_XBOX = 16384;            // one TMA box: 64 rows x 16 complex or 32 real columns
constexpr int GZ_XSLOT = 2 * GZ_XBOX;     // both blocks of a pivot

// TMA: a narrow pivot (one 64-position tile, blocks of at most 16 complex or
// 32 real columns) whose rows arrive by tiled TMA copies (xmap) into two
// chunk slots of shared memory, the next chunk's copy in flight while the
// current one is turned into digits; otherwise the builders read G directly.
template <bool CPLX, bool TMA>
__global__ void __launch_bounds__(GZ_THREADS, 1) gram_ozaki_kernel(
    const __grid_constant__ CUtensorMap xmap,
    const double *__restrict__ G, int64_t ld, int64_t m, const int32_t *__restrict__ pairs,
    const int32_t *__restrict__ cexp, unsigned long long *__restrict__ acc_out, int k2max,
    int rows_per_block, unsigned long long *__restrict__ counters, StepCtl ctl) {
    extern __shared__ __align__(1024) uint8_t oz_smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) unsigned long long bar_mma[2];
    __shared__ __align__(8) unsigned long long bar_x[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int sexp[kOzMaxK2];
    __shared__ int s_abort;

    const int32_t *pd = pairs + 4 * blockIdx.y;
    if (ctl.mod_step) {
        const bool skip = pair_skip_decide(ctl, pd, blockIdx.y);
        if (blockIdx.x == 0 && blockIdx.z == 0 && threadIdx.x == 0)
            ctl.flags[blockIdx.y] = skip ? kPairSkipped : 0;
        if (skip) return;
    }
    const int k = pd[1] + pd[3];
    const int K2 = CPLX ? 2 * k : k;
    // tile pair (ta, tb) of this block: blockIdx.z = tb (tb + 1) / 2 + ta
    int ta = blockIdx.z, tb = 0;
    while (ta > tb) {
        ta -= tb + 1;
        ++tb;
    }
    if (64 * tb >= K2) return;
    const bool offd = ta != tb;
    const int pa0 = 64 * ta, pb0 = 64 * tb;  // first positions of the A and B tiles
    const int NP = (min(64, K2 - pb0) + 15) & ~15;  // N of the MMA (multiple of 16)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    m = pair_rows(ctl, blockIdx.y, m);
    const int64_t row0 = (int64_t)blockIdx.x * rows_per_block;
    if (row0 >= m) return;
    const int64_t row1 = min((int64_t)m, row0 + rows_per_block);

    if (tid == 0) s_abort = 0;
    for (int a = tid; a < K2; a += GZ_THREADS) {
        const int c = CPLX ? (a < k ? a : a - k) : a;
        sexp[a] = cexp[c < pd[1] ? pd[0] + c : pd[2] + (c - pd[1])];
    }
    if (warp == 0) tmem_alloc(su32(&tmem_base_sh), 512);
    if (tid == 0) {
        mbar_init(su32(&bar_mma[0]), 1);
        mbar_init(su32(&bar_mma[1]), 1);
        mbar_init(su32(&bar_x[0]), 1);
        mbar_init(su32(&bar_x[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // operand rows beyond K2 of a partial last tile stay zero for every chunk
    if (K2 - pb0 < 64)
        for (int i = tid; i < 2 * GZ_BUF_BYTES / 16; i += GZ_THREADS)
            reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const uint32_t idesc = idesc_f16(64, NP);

    // this thread: TMEM lane (warp%4)*32 + lane holds output row (warp%4)*16 + lane
    // for lane < 16 (M = 64 layout); columns [cq*16, cq*16 + 16)
    const int quad = warp & 3, cq = warp >> 2;
    const int orow = quad * 16 + lane;
    const bool owns = lane < 16 && pa0 + orow < K2;
    long long w0[16], w1[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        w0[j] = 0;
        w1[j] = 0;
    }
    uint32_t ph[2] = {0u, 0u};
    bool pending[2] = {false, false};
    const uint32_t sbase = su32(sm);
    const int nsc = (int)((row1 - row0 + GZ_KC - 1) / GZ_KC);

    // One thread polls the mbarrier; the others wait in the block barrier that
    // follows (spinning threads would take issue slots from the digit builders).
    // A wait that runs out leaves the buffer pending, so that the teardown
    // still waits for its products before the TMEM is freed.
    auto wait_buf = [&](int b, uint64_t limit) {
        if (!pending[b]) return;
        const int ok = __syncthreads_and(tid != 0 || mbar_wait(su32(&bar_mma[b]), ph[b], limit));
        if (ok) {
            ph[b] ^= 1u;
            pending[b] = false;
        } else {
            s_abort = 1;
        }
    };
    // digits of rows [row0 + 64 i, +64) of the 64 positions from pos0 into
    // buffer b, by warps 1..15 (warp 0 issues the tensor-core products meanwhile);
    // item -> (column a, row pair): rows l, l+1 packed into one 32-bit store.
    // Two items per thread at a time, loads first (the 64 accumulator
    // registers of the drain leave no room for more).
    constexpr int GZ_BUILDERS = GZ_THREADS - 32;
    constexpr int GZ_NITEMS = 64 * (GZ_KC / 2);
    auto build = [&](int i, int b, int pos0) {
        const int64_t c0 = row0 + (int64_t)i * GZ_KC;
        const int nrow = (int)min((int64_t)GZ_KC, row1 - c0);
        uint8_t *buf = sm + (size_t)b * GZ_BUF_BYTES;
        for (int base = tid - 32; base < GZ_NITEMS; base += 2 * GZ_BUILDERS) {
            double xv0[2], xv1[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = base + u * GZ_BUILDERS;
                const int a = pos0 + idx / (GZ_KC / 2);
                const int lp = (idx % (GZ_KC / 2)) * 2;
                xv0[u] = 0.0;
                xv1[u] = 0.0;
                if (idx < GZ_NITEMS && a < K2) {
                    const int c = CPLX ? (a < k ? a : a - k) : a;
                    const int64_t col = c < pd[1] ? (int64_t)pd[0] + c : (int64_t)pd[2] + (c - pd[1]);
                    const int ri = (CPLX && a >= k) ? 1 : 0;
                    if (lp < nrow) xv0[u] = CPLX ? G[(col * ld + c0 + lp) * 2 + ri] : G[col * ld + c0 + lp];
                    if (lp + 1 < nrow)
                        xv1[u] = CPLX ? G[(col * ld + c0 + lp + 1) * 2 + ri] : G[col * ld + c0 + lp + 1];
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = base + u * GZ_BUILDERS;
                const int a = pos0 + idx / (GZ_KC / 2);
                const int lp = (idx % (GZ_KC / 2)) * 2;
                if (idx >= GZ_NITEMS || a >= K2) continue;
                const int e = sexp[a];
                const unsigned long long q0 = fixed63(xv0[u], e), q1 = fixed63(xv1[u], e);
                const bool n0 = neg_bits(xv0[u]), n1 = neg_bits(xv1[u]);
                const uint32_t off = sw128_off(a - pos0, lp * 2);
#pragma unroll
                for (int t = 1; t <= GZ_SLICES; ++t)
                    *reinterpret_cast<uint32_t *>(buf + (t - 1) * GZ_SLICE_BYTES + off) =
                        dg_digits2_bits(q0, n0, q1, n1, t);
            }
        }
    };

    // TMA: chunk j (rows row0 + 64 j ..) into slot j & 1, issued by thread 0
    // once the slot's previous chunk has been turned into digits
    uint8_t *sX = sm + 2 * GZ_BUF_BYTES;
    constexpr int XBOXC = CPLX ? 16 : 32;  // columns per box
    int x_last[2] = {-1, -1};              // last chunk issued into each slot (thread 0)
    auto issue_x = [&](int j) {
        if (!TMA || tid != 0 || j >= nsc) return;
        const int slot = j & 1;
        const uint32_t bar = su32(&bar_x[slot]);
        const uint32_t dst = su32(sX) + (uint32_t)(slot * GZ_XSLOT);
        const int y = (int)((CPLX ? 2 : 1) * (row0 + (int64_t)j * GZ_KC));
        mbar_expect_tx(bar, (uint32_t)(((pd[1] > 0) + (pd[3] > 0)) * GZ_XBOX));
        if (pd[1] > 0) tma_load_2d(dst, &xmap, y, pd[0], bar);
        if (pd[3] > 0) tma_load_2d(dst + GZ_XBOX, &xmap, y, pd[2], bar);
        x_last[slot] = j;
    };
    // digits of chunk i from its slot: an item is one pivot column and a row
    // pair (complex: both of its positions, Re at c and Im at c + k)
    auto build_x = [&](int i, int b) {
        const int slot = i & 1;
        if (!mbar_wait(su32(&bar_x[slot]), (uint32_t)((i >> 1) & 1), ctl.wait_ns)) {
            s_abort = 1;
            return;
        }
        const int64_t c0 = row0 + (int64_t)i * GZ_KC;
        const int nrow = (int)min((int64_t)GZ_KC, row1 - c0);
        uint8_t *buf = sm + (size_t)b * GZ_BUF_BYTES;
        const uint8_t *xs = sX + (size_t)slot * GZ_XSLOT;
        constexpr int NIT = (CPLX ? 32 : 64) * (GZ_KC / 2);
        for (int idx = tid - 32; idx < NIT; idx += GZ_THREADS - 32) {
            const int c = idx / (GZ_KC / 2);
            const int lp = (idx % (GZ_KC / 2)) * 2;
            if (c >= k) continue;
            const int cs = c < pd[1] ? c : XBOXC + (c - pd[1]);
            const bool in0 = lp < nrow, in1 = lp + 1 < nrow;
            if (CPLX) {
                const double2 *col = reinterpret_cast<const double2 *>(xs + (size_t)cs * (GZ_KC * 16));
                const double2 z0 = in0 ? col[lp] : make_double2(0.0, 0.0);
                const double2 z1 = in1 ? col[lp + 1] : make_double2(0.0, 0.0);
                const int e = sexp[c];  // the same for Re and Im
                const unsigned long long r0 = fixed63(z0.x, e), r1 = fixed63(z1.x, e);
                const unsigned long long i0 = fixed63(z0.y, e), i1 = fixed63(z1.y, e);
                const bool nr0 = neg_bits(z0.x), nr1 = neg_bits(z1.x), ni0 = neg_bits(z0.y), ni1 = neg_bits(z1.y);
                const uint32_t offr = sw128_off(c, lp * 2), offi = sw128_off(c + k, lp * 2);
#pragma unroll
                for (int t = 1; t <= GZ_SLICES; ++t) {
                    uint8_t *tile = buf + (t - 1) * GZ_SLICE_BYTES;
                    *reinterpret_cast<uint32_t *>(tile + offr) = dg_digits2_bits(r0, nr0, r1, nr1, t);
                    *reinterpret_cast<uint32_t *>(tile + offi) = dg_digits2_bits(i0, ni0, i1, ni1, t);
                }
            } else {
                const double *col = reinterpret_cast<const double *>(xs + (size_t)cs * (GZ_KC * 8));
                const double x0 = in0 ? col[lp] : 0.0, x1 = in1 ? col[lp + 1] : 0.0;
                const int e = sexp[c];
                const unsigned long long q0 = fixed63(x0, e), q1 = fixed63(x1, e);
                const bool n0 = neg_bits(x0), n1 = neg_bits(x1);
                const uint32_t off = sw128_off(c, lp * 2);
#pragma unroll
                for (int t = 1; t <= GZ_SLICES; ++t)
                    *reinterpret_cast<uint32_t *>(buf + (t - 1) * GZ_SLICE_BYTES + off) =
                        dg_digits2_bits(q0, n0, q1, n1, t);
            }
        }
    };

    // For each A digit t, the B tiles of digits u, u + 1, ... are adjacent in
    // shared memory and their diagonals t + u, t + u + 1, ... are adjacent
    // 64-column groups in TMEM: one product with N = 64 * run covers a run of
    // up to four (rows of a digit tile beyond K2 are zero, so the columns
    // beyond K2 of each group receive zeros). Digit t = 1 meets every diagonal
    // once, so its products (accumulate = 0 in the first chunk of a 128-row
    // accumulation) initialize all groups. One thread issues.
    auto issue = [&](uint32_t abase, uint32_t bbase, bool first) {
        for (int t = 1; t <= GZ_SLICES; ++t) {
            const int umax = GZ_SLICES + 1 - t;
            const uint32_t a0 = abase + (uint32_t)((t - 1) * GZ_SLICE_BYTES);
            for (int u = 1; u <= umax;) {
                // adjacent tiles in one product (only when a tile has no
                // padding rows, which a wider N would multiply)
                const int run = NP == 64 ? min(4, umax - u + 1) : 1;
                const uint32_t id = run == 1 ? idesc : idesc_f16(64, 64 * run);
                const uint32_t dt = tmem + (uint32_t)((t + u - 2) * 64);
                const uint32_t b0 = bbase + (uint32_t)((u - 1) * GZ_SLICE_BYTES);
#pragma unroll
                for (int ks = 0; ks < GZ_KC / 16; ++ks)
                    mma_f16(dt, desc_sw128(a0 + ks * 32), desc_sw128(b0 + ks * 32), id,
                            (first && t == 1 && ks == 0) ? 0u : 1u);
                u += run;
            }
        }
    };
    // every group of the last 128 rows into the two int64 words of each output
    auto drain = [&]() {
        // two groups (32 columns of this thread) per TMEM round trip
#pragma unroll
        for (int d0 = 2; d0 <= GZ_SLICES + 1; d0 += 2) {
            uint32_t v[4][8];
#pragma unroll
            for (int g = 0; g < 2; ++g)
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    tmem_ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)((d0 + g - 2) * 64 + cq * 16 + 8 * h),
                             v[2 * g + h]);
            tmem_wait_ld();
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int sh = kBeta * (GZ_SLICES + 1 - (d0 + g));
                const long long mul = 1ll << (sh & 31);
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int iv = __float2int_rn(__uint_as_float(v[2 * g + h][j]));  // exact, |v| < 2^24
                        if (sh >= 32)
                            w1[8 * h + j] += (long long)iv * mul;
                        else
                            w0[8 * h + j] += (long long)iv * mul;
                    }
            }
        }
    };

    if (!offd) {
        // diagonal tile: one operand tile serves as A and B; two buffers, the
        // digits of the next 64 rows built while the products read the current
        if (TMA) {
            issue_x(0);
            issue_x(1);
        }
        if (nsc > 0 && warp != 0) {
            if (TMA)
                build_x(0, 0);
            else
                build(0, 0, pa0);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        issue_x(2);  // chunk 0's slot has been read
        for (int i = 0; i < nsc && !s_abort; ++i) {
            const int b = i & 1;
            const bool first = (i & 1) == 0;  // first 64 rows of a 128-row accumulation
            if (tid == 0) {
                const uint32_t base = sbase + (uint32_t)(b * GZ_BUF_BYTES);
                issue(base, base, first);
                mma_commit(su32(&bar_mma[b]));
            }
            pending[b] = true;
            if (i + 1 < nsc) {
                wait_buf(b ^ 1, ctl.wait_ns);  // the products that read the other buffer are done
                if (warp != 0) {
                    if (TMA)
                        build_x(i + 1, b ^ 1);
                    else
                        build(i + 1, b ^ 1, pa0);
                }
                fence_async_smem();
            }
            if ((i & 1) == 1 || i == nsc - 1) {
                wait_buf(b ^ 1, ctl.wait_ns);
                wait_buf(b, ctl.wait_ns);
                tc_fence_after();
                if (!s_abort) drain();
                tc_fence_before();
            }
            __syncthreads();
            tc_fence_after();
            issue_x(i + 3);  // chunk i + 1's slot has been read
        }
    } else {
        // off-diagonal tile: A digits in buffer 0, B digits in buffer 1
        for (int i = 0; i < nsc && !s_abort; ++i) {
            const bool first = (i & 1) == 0;
            wait_buf(0, ctl.wait_ns);  // the previous chunk's products have read both buffers
            if (s_abort) break;
            if (warp != 0) {
                build(i, 0, pa0);
                build(i, 1, pb0);
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
                issue(sbase, sbase + (uint32_t)GZ_BUF_BYTES, first);
                mma_commit(su32(&bar_mma[0]));
            }
            pending[0] = true;
            if ((i & 1) == 1 || i == nsc - 1) {
                wait_buf(0, ctl.wait_ns);
                tc_fence_after();
                if (!s_abort) drain();
                tc_fence_before();
            }
            __syncthreads();
            tc_fence_after();
        }
    }
    if (s_abort) {
        // in-flight products finish before the TMEM is freed (the default bound:
        // the products still complete after a shorter wait ran out)
        wait_buf(0, kWaitLimitNs);
        wait_buf(1, kWaitLimitNs);
        if (tid == 0 && counters) atomicOr(&counters[kCntErr], kErrTimeout);
    } else if (owns) {
        // add the partial sums: acc_out[pair][col b][row a] = {lo, hi}
        unsigned long long *dst = acc_out + (size_t)blockIdx.y * k2max * k2max * 2;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int bcol = pb0 + cq * 16 + j;
            if (bcol < K2) {
                // T = w0 + w1 * 2^32 as (lo, hi)
                const unsigned long long l1 = (unsigned long long)w1[j] << 32;
                const long long h1 = w1[j] >> 32;
                const unsigned long long lo = (unsigned long long)w0[j] + l1;
                const long long hi = (w0[j] >> 63) + h1 + (lo < l1 ? 1 : 0);
                unsigned long long *w = dst + ((size_t)bcol * k2max + pa0 + orow) * 2;
                const unsigned long long old = atomicAdd(w, lo);
                const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
                atomicAdd(w + 1, (unsigned long long)hi + carry);
            }
        }
    }
    // chunk copies still in flight (after a wait ran out) land before the
    // shared memory is released
    if (TMA && tid == 0)
        for (int sl = 0; sl < 2; ++sl)
            if (x_last[sl] >= 0) mbar_wait(su32(&bar_x[sl]), (uint32_t)((x_last[sl] >> 1) & 1), kWaitLimitNs);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// int128 fixed-point Gram -> FP64 A_P (complex: Re = C11 + C22, Im = C12 - C21),
// value = acc * 2^(e_a + e_b - 7 (s + 1)); both triangles written.
template <bool CPLX>
__global__ void __launch_bounds__(256) gram_fixed_to_double_kernel(
    const unsigned long long *__restrict__ acc, const int32_t *__restrict__ pairs,
    const int32_t *__restrict__ cexp, double *__restrict__ A, int kmax, int k2max, int slices) {
    const int32_t *pd = pairs + 4 * blockIdx.y;
    const int k = pd[1] + pd[3];
    const int idx = blockIdx.x * 256 + threadIdx.x;
    if (idx >= k * k) return;
    const int a = idx % k, b = idx / k;
    const unsigned long long *P = acc + (size_t)blockIdx.y * k2max * k2max * 2;
    // only the tiles (ta, tb) with ta <= tb (64 positions each) are formed: a
    // lower one is read as the transpose
    auto ld128 = [&](int r, int c, unsigned long long &lo, long long &hi) {
        if ((r >> 6) > (c >> 6)) {
            const int x = r;
            r = c;
            c = x;
        }
        lo = P[((size_t)c * k2max + r) * 2];
        hi = (long long)P[((size_t)c * k2max + r) * 2 + 1];
    };
    auto add = [](unsigned long long &lo, long long &hi, unsigned long long lo2, long long hi2, bool sub) {
        if (sub) {  // negate (lo2, hi2)
            lo2 = ~lo2 + 1ull;
            hi2 = ~hi2 + (lo2 == 0ull ? 1 : 0);
        }
        const unsigned long long l = lo + lo2;
        hi = hi + hi2 + (l < lo ? 1 : 0);
        lo = l;
    };
    auto to_double = [](unsigned long long lo, long long hi) {
        // hi * 2^64 + lo (lo unsigned), rounded to double
        return fma((double)hi, 18446744073709551616.0, (double)lo);
    };
    const int ca = a < pd[1] ? pd[0] + a : pd[2] + (a - pd[1]);
    const int cb = b < pd[1] ? pd[0] + b : pd[2] + (b - pd[1]);
    const int ex = cexp[ca] + cexp[cb] - kBeta * (slices + 1);
    const double scale = ldexp(1.0, ex);
    double *Ap = A + (size_t)blockIdx.y * kmax * kmax * (CPLX ? 2 : 1);
    if (CPLX) {
        unsigned long long rl, l2;
        long long rh, h2;
        ld128(a, b, rl, rh);
        ld128(a + k, b + k, l2, h2);
        add(rl, rh, l2, h2, false);
        unsigned long long il;
        long long ih;
        ld128(a, b + k, il, ih);
        ld128(a + k, b, l2, h2);
        add(il, ih, l2, h2, true);
        Ap[((size_t)b * kmax + a) * 2] = to_double(rl, rh) * scale;
        Ap[((size_t)b * kmax + a) * 2 + 1] = to_double(il, ih) * scale;
    } else {
        unsigned long long rl;
        long long rh;
        ld128(a, b, rl, rh);
        Ap[(size_t)b * kmax + a] = to_double(rl, rh) * scale;
    }
}

template <typename K>
cudaError_t set_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

int ozaki_default_slices(bool gram) { return gram ? GZ_SLICES : kUdMaxSlices; }

bool ozaki_supported(bool cplx, int kmax) { return (cplx ? 2 * kmax : kmax) <= kOzMaxK2; }

size_t ozaki_gram_workspace_bytes(int npairs, int kmax, bool cplx) {
    const int k2 = cplx ? 2 * kmax : kmax;
    return (size_t)npairs * k2 * k2 * 2 * sizeof(unsigned long long);
}

cudaError_t launch_colexp(bool cplx, const double *G, int64_t ld, int64_t m, int64_t n,
                          int32_t *cexp, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (cplx)
        colexp_kernel<true><<<(unsigned)n, 256, 0, st>>>(G, ld, m, cexp);
    else
        colexp_kernel<false><<<(unsigned)n, 256, 0, st>>>(G, ld, m, cexp);
    return cudaGetLastError();
}

cudaError_t launch_colexp_pairs(bool cplx, const double *G, int64_t ld, int64_t m,
                                const int32_t *pairs, int npairs, int kmax, int32_t *cexp,
                                cudaStream_t st, StepCtl ctl) {
    if (npairs <= 0) return cudaSuccess;
    dim3 grid((unsigned)kmax, npairs);
    if (cplx)
        colexp_pairs_kernel<true><<<grid, 256, 0, st>>>(G, ld, m, pairs, cexp, ctl);
    else
        colexp_pairs_kernel<false><<<grid, 256, 0, st>>>(G, ld, m, pairs, cexp, ctl);
    return cudaGetLastError();
}

// Gram by digit products: cexp must hold the column exponents of G (launch_colexp);
// acc (ozaki_gram_workspace_bytes) is zeroed here; A receives the FP64 blocks.
cudaError_t launch_gram_ozaki(bool cplx, const double *G, int64_t ld, int64_t m, int64_t ncols,
                              const int32_t *pairs, int npairs, double *A, int kmax, int maxblk,
                              const int32_t *cexp, unsigned long long *acc, int slices,
                              unsigned long long *counters, cudaStream_t st, StepCtl ctl) {
    if (npairs <= 0) return cudaSuccess;
    const int k2max = cplx ? 2 * kmax : kmax;
    if (k2max > kOzMaxK2 || slices != GZ_SLICES) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(acc, 0, ozaki_gram_workspace_bytes(npairs, kmax, cplx), st);
    if (e != cudaSuccess) return e;
    // tile pairs of the widest pivot (upper triangle of T x T tiles of 64)
    const int T = (k2max + 63) / 64;
    const int ntp = T * (T + 1) / 2;
    // rows per block: 512 (measured: 512 and 640 rows balance the waves of
    // 1-per-SM blocks best at m = 4096), fewer when that leaves the GPU idle;
    // a multiple of 128 rows
    int rpb = 2 * GZ_KC * 4;
    while (rpb > 2 * GZ_KC && (int64_t)npairs * ntp * ((m + rpb - 1) / rpb) < 2 * 152) rpb /= 2;
    dim3 grid((unsigned)((m + rpb - 1) / rpb), npairs, ntp);
    // narrow pivots whose blocks fit a box, on 16-byte aligned rows: chunks by TMA
    const int E = cplx ? 2 : 1;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    const bool tma = T == 1 && maxblk > 0 && maxblk <= (cplx ? 16 : 32) && ((uintptr_t)G & 15) == 0 &&
                     ((ld * E * 8) & 15) == 0 && ncols >= 1 && ld * E < (1ll << 31) &&
                     encode_x_map(&map, cplx, G, ld, m, ncols, GZ_KC, cplx ? 16 : 32);
    const size_t smem = (size_t)2 * GZ_BUF_BYTES + (tma ? 2 * (size_t)GZ_XSLOT : 0) + 1024;
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e2 = set_smem(kern, smem);
        if (e2 != cudaSuccess) return e2;
        kern<<<grid, GZ_THREADS, smem, st>>>(map, G, ld, m, pairs, cexp, acc, k2max, rpb, counters, ctl);
        return cudaSuccess;
    };
    if (cplx)
        e = tma ? run(gram_ozaki_kernel<true, true>) : run(gram_ozaki_kernel<true, false>);
    else
        e = tma ? run(gram_ozaki_kernel<false, true>) : run(gram_ozaki_kernel<false, false>);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 g2((unsigned)((kmax * kmax + 255) / 256), npairs);
    if (cplx)
        gram_fixed_to_double_kernel<true><<<g2, 256, 0, st>>>(acc, pairs, cexp, A, kmax, k2max, slices);
    else
        gram_fixed_to_double_kernel<false><<<g2, 256, 0, st>>>(acc, pairs, cexp, A, kmax, k2max, slices);
    return cudaGetLastError();
}

}  // namespace jj
