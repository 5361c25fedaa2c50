// Internal declarations shared by the CUDA translation units of libjjacobi.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/jjacobi.h"
#include "../../include/jjacobi_kernels.h"

namespace jj {

// Error flags accumulated on the device (counters[2]).
constexpr unsigned long long kErrNotPosdef = 1ull;
constexpr unsigned long long kErrNonfinite = 2ull;
constexpr unsigned long long kErrTimeout = 4ull;

// 128 * 2^-53: the convergence threshold of the published workloads.
constexpr double kDefaultTol = 128.0 * 1.1102230246251565404e-16;

// Counter slots.
enum { kCntRot = 0, kCntMaxOff = 1, kCntErr = 2, kCntPairs = 3, kCntPairsRot = 4, kNumCounters = 8 };

// Parameters of one J-unitary rotation on a column pair (g_r, g_s), in the form
//   g_r' = ce * g_r - hs * g_s,   g_s' = se * g_r + c * g_s
// with ce = c e^{i alpha}, se = s e^{i alpha}, hs = hyp * s (Alg. 3.1, (2.3)).
struct Rot {
    double ce_re, ce_im, se_re, se_im, c, hs;
    double dr, ds;  // updated diagonal a_rr', a_ss'
};

// Rotation of Alg. 3.1 for the pivot (a_rr, a_ss, a_rs), hyp = J_rr J_ss.
//   eta = sgn(Re a_rs) |a_rs|, e^{i alpha} = a_rs / eta (real: eta = a_rs);
//   theta = hyp (a_ss - hyp a_rr) / (2 eta);
//   t = sgn(theta) / (|theta| + sqrt(theta^2 + hyp)), or 1/(2 theta) when
//   |theta| > 1e150; c = 1/sqrt(1 + hyp t^2), s = c t;
//   a_rr' = a_rr - hyp t eta, a_ss' = a_ss + t eta.
// hyp = +J_rr J_ss is the reading of the printed sign that keeps W_P
// J-unitary; sgn(0) = +1. Returns false when the hyperbolic case has
// theta^2 < 1 (the pair is not positive definite in working precision).
__device__ __forceinline__ bool rotation(double arr, double ass, double are, double aim,
                                         int hyp, bool cplx, Rot &o) {
    const double absa = cplx ? sqrt(are * are + aim * aim) : fabs(are);
    const double eta = are >= 0.0 ? absa : -absa;
    double er = 1.0, ei = 0.0;
    if (cplx) {
        const double inv = 1.0 / eta;
        er = are * inv;
        ei = aim * inv;
    }
    const double h = (double)hyp;
    const double theta = h * (ass - h * arr) / (2.0 * eta);
    const double at = fabs(theta);
    double t;
    if (at > 1e150) {
        t = 0.5 / theta;
    } else {
        const double rad = theta * theta + h;
        if (!(rad >= 0.0)) return false;
        t = 1.0 / (at + sqrt(rad));
        if (theta < 0.0) t = -t;
    }
    const double q = 1.0 + h * t * t;
    if (!(q > 0.0)) return false;
    const double c = 1.0 / sqrt(q);
    const double s = c * t;
    o.c = c;
    o.hs = h * s;
    o.ce_re = c * er;
    o.ce_im = c * ei;
    o.se_re = s * er;
    o.se_im = s * ei;
    o.dr = arr - h * t * eta;
    o.ds = ass + t * eta;
    return true;
}

// Apply a rotation to one row entry of a complex column pair.
__device__ __forceinline__ void rot_apply_c(const Rot &R, double &xr, double &xi, double &yr,
                                            double &yi) {
    const double nxr = fma(R.ce_re, xr, fma(-R.ce_im, xi, -R.hs * yr));
    const double nxi = fma(R.ce_re, xi, fma(R.ce_im, xr, -R.hs * yi));
    const double nyr = fma(R.se_re, xr, fma(-R.se_im, xi, R.c * yr));
    const double nyi = fma(R.se_re, xi, fma(R.se_im, xr, R.c * yi));
    xr = nxr;
    xi = nxi;
    yr = nyr;
    yi = nyi;
}

__device__ __forceinline__ void rot_apply_r(const Rot &R, double &x, double &y) {
    const double nx = fma(R.ce_re, x, -R.hs * y);
    const double ny = fma(R.se_re, x, R.c * y);
    x = nx;
    y = ny;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v) {
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// Skipping unchanged pivot pairs. A pair (i, j) whose two blocks have not
// changed since the pair was last found diagonal (its inner solve applied no
// rotation) would produce the same Gram and again no rotation: the kernels are
// deterministic (the split-precision Gram adds exact integers), so skipping it
// is exact. Stamps are global step indices T = sweep * steps + step.
struct StepCtl {
    int32_t *mod_step = nullptr;      // [n]: by block start column, step of the last change (-1: never)
    int32_t *clean_at = nullptr;      // [slots]: step when the slot was found clean (-1: not)
    int32_t *flags = nullptr;         // [npairs]: bit 0 skipped, bit 1 identity (no rotation)
    const int32_t *sweep = nullptr;   // device sweep counter (1 in the first sweep)
    int step = 0;                     // position of this step in the sweep
    int steps = 0;                    // steps per sweep
    int npairs = 0;                   // pairs in this step
    int slot_base = 0;                // clean_at index of pair 0 of this step
    // Several independent problems in one work matrix (batched solve):
    const int32_t *rows = nullptr;    // [npairs]: rows of the pair's problem (nullptr: all m)
    const int32_t *prob = nullptr;    // [npairs]: problem of the pair
    unsigned long long *prob_rot = nullptr;  // [2 problems]: rotations, error flags (this sweep)
    // [npairs][2]: bit c set when the inner solve rotated column c of the pair
    // (columns never rotated keep W's column e_c, so the update can skip them)
    unsigned long long *touched = nullptr;
    // bound of every device-side wait of the step's kernels (nanoseconds)
    unsigned long long wait_ns = 2000000000ull;
};
constexpr int kPairSkipped = 1;
constexpr int kPairIdentity = 2;

// Operand of the split-precision update: the fp16 digits of D (W2 - I) as
// shared-memory images (SWIZZLE_128B, K-major: 64 rows of 128 bytes per
// digit, row j = output position j, K position a = row of W2, on the
// real-form positions of jj_digits.cuh), and their column exponents, one
// image per 64 x 64 tile (kc, nc) of a wide pivot (T tiles per side, T = 1 up
// to 64 real-form positions; the inner solve builds the image of such a
// pivot itself, launch_wimage the others). D holds the column exponents of
// the pivot columns (cexp). Used only when the update runs as digit products.
struct UpdDigits {
    uint8_t *img = nullptr;        // [npairs][T][T][slices][64 * 128]
    int32_t *wexp = nullptr;       // [npairs][T][T][64]
    const int32_t *cexp = nullptr; // column exponents of G (by work column)
    int slices = 0;
};
constexpr int kUpdSliceBytes = 64 * 128;
constexpr int kUdMaxSlices = 11;  // balanced 8-bit digits per operand of the update (88 bits)
constexpr int kUdMaxTiles = 4;    // 64-position tiles per pivot side (256 real-form positions)

// Decide (Gram kernels) whether pair q of this step can be skipped: the slot was
// found clean at step `clean` and neither block changed after it.
__device__ __forceinline__ bool pair_skip_decide(const StepCtl &c, const int32_t *pd, int q) {
    if (!c.mod_step) return false;
    const int clean = c.clean_at[c.slot_base + q];
    return clean >= 0 && c.mod_step[pd[0]] < clean && c.mod_step[pd[2]] < clean;
}

// Bookkeeping after the inner solve of pair q (one thread).
__device__ __forceinline__ void pair_record(const StepCtl &c, const int32_t *pd, int q,
                                            bool rotated, bool failed) {
    if (!c.mod_step) return;
    const int T = (*c.sweep) * c.steps + c.step;
    if (rotated) {
        c.mod_step[pd[0]] = T;
        c.mod_step[pd[2]] = T;
        c.clean_at[c.slot_base + q] = -1;
        c.flags[q] = 0;
    } else {
        c.clean_at[c.slot_base + q] = failed ? -1 : T;
        c.flags[q] = kPairIdentity;
    }
}

// Rotations and error flags of pair q credited to its problem (batched solve):
// prob_rot[2 p] rotations, prob_rot[2 p + 1] error flags.
__device__ __forceinline__ void pair_count_prob(const StepCtl &c, int q, unsigned long long rot) {
    if (c.prob_rot && rot) atomicAdd(&c.prob_rot[2 * c.prob[q]], rot);
}
__device__ __forceinline__ void pair_flag_prob(const StepCtl &c, int q, unsigned long long flag) {
    if (c.prob_rot) atomicOr(&c.prob_rot[2 * c.prob[q] + 1], flag);
}

// Rows of the problem that pair q belongs to.
__device__ __forceinline__ int64_t pair_rows(const StepCtl &c, int q, int64_t m) {
    return c.rows ? (int64_t)c.rows[q] : m;
}

__device__ __forceinline__ bool pair_passthrough(const StepCtl &c, int q) {
    return c.flags && (c.flags[q] & (kPairSkipped | kPairIdentity));
}

// ---------------------------------------------------------------------------
// Launchers (host functions, defined in the .cu files)
// ---------------------------------------------------------------------------
cudaError_t launch_column_norms(bool cplx, const double *G, int64_t ld, int64_t m, int64_t n,
                                double *d, cudaStream_t st);
cudaError_t launch_plain_step(bool cplx, double *G, int64_t ld, int64_t m, int64_t n,
                              const int32_t *pairs, int npairs, const int8_t *J, double *d,
                              double tol, unsigned long long *counters, cudaStream_t st);
cudaError_t launch_extract(bool cplx, const double *G, int64_t ld, int64_t m, int64_t n,
                           const int8_t *J, const int32_t *perm, double *lambda, double *U,
                           int64_t ldu, cudaStream_t st);
// Gw[:, c] = G[:, src[c]] (gather) or G[:, src[c]] = Gw[:, c] (scatter).
cudaError_t launch_permute_columns(bool cplx, const double *A, int64_t lda, double *B,
                                   int64_t ldb, int64_t m, int64_t n, const int32_t *perm,
                                   bool scatter, cudaStream_t st);

cudaError_t launch_gram(bool cplx, int gemm, const double *G, int64_t ld, int64_t m,
                        const int32_t *pairs, int npairs, double *A, int kmax,
                        cudaStream_t st, StepCtl ctl = StepCtl());
cudaError_t launch_inner(bool cplx, double *A, double *W, int kmax, const int32_t *pairs,
                         int npairs, const int8_t *J, double tol, int inner_max_sweeps,
                         int inner_block, unsigned long long *counters, cudaStream_t st,
                         StepCtl ctl = StepCtl(), UpdDigits ud = UpdDigits(), int pass = 0,
                         bool special = false);
cudaError_t launch_update(bool cplx, int gemm, const double *Gs, double *Gd, int64_t ld,
                          int64_t m, const int32_t *pairs, int npairs, const double *W,
                          int kmax, cudaStream_t st, StepCtl ctl = StepCtl());

// Whether the inner solve can run single passes (block-oriented strategy).
bool inner_single_pass_supported(bool cplx, int kmax);

// Split-precision (fp16 digit) forms on the tensor cores (jj_ozaki.cu).
int ozaki_default_slices(bool gram);
bool ozaki_supported(bool cplx, int kmax);
size_t ozaki_gram_workspace_bytes(int npairs, int kmax, bool cplx);
cudaError_t launch_colexp(bool cplx, const double *G, int64_t ld, int64_t m, int64_t n,
                          int32_t *cexp, cudaStream_t st);
// Column exponents of the pivot columns of one step's pairs (grid kmax x npairs).
cudaError_t launch_colexp_pairs(bool cplx, const double *G, int64_t ld, int64_t m,
                                const int32_t *pairs, int npairs, int kmax, int32_t *cexp,
                                cudaStream_t st, StepCtl ctl);
// ncols: columns of G; maxblk: the largest block of any pair (0: unknown):
// narrow pivots whose blocks fit a TMA box take their rows by TMA.
cudaError_t launch_gram_ozaki(bool cplx, const double *G, int64_t ld, int64_t m, int64_t ncols,
                              const int32_t *pairs, int npairs, double *A, int kmax, int maxblk,
                              const int32_t *cexp, unsigned long long *acc, int slices,
                              unsigned long long *counters, cudaStream_t st,
                              StepCtl ctl = StepCtl());
// Split-precision block update (jj_update_digits.cu): ud.img / ud.wexp hold the
// W-side digits of every active pair (built by the inner solve, or by
// launch_wimage), cexp the column exponents of Gs, scratch
// ud_scratch_bytes(nctas, ud_max_tiles(cplx, kmax)) bytes; nctas persistent
// blocks (ud_num_ctas()).
// ncols: columns of Gs (the extent the narrow kernel's tensor map covers);
// maxblk: the largest block of any pair (0: unknown). Narrow pivots whose
// blocks fit a TMA box run update_narrow_kernel (jj_update_narrow.cu), the
// others update_digits_kernel.
cudaError_t launch_update_digits(bool cplx, const double *Gs, double *Gd, int64_t ld, int64_t m,
                                 int64_t ncols, const int32_t *pairs, int npairs, int kmax, int maxblk,
                                 const int32_t *cexp, const UpdDigits &ud, long long *scratch, int nctas,
                                 unsigned long long *counters, cudaStream_t st,
                                 StepCtl ctl = StepCtl());
bool un_supported(bool cplx, const double *Gs, int64_t ld, int64_t m, int64_t ncols, int kmax, int maxblk);
// Tensor map of a column-major work matrix (complex interleaved) as a 2-D array
// of doubles: E m x ncols with row stride ld E; boxes of box_rows rows of
// box_cols columns. False when the driver's encoder is unavailable or refuses.
bool encode_x_map(CUtensorMap *map, bool cplx, const double *G, int64_t ld, int64_t m, int64_t ncols,
                  int box_rows, int box_cols);
cudaError_t launch_update_narrow(bool cplx, const double *Gs, double *Gd, int64_t ld, int64_t m, int64_t ncols,
                                 const int32_t *pairs, int npairs, const int32_t *cexp, const UpdDigits &ud,
                                 int nctas, unsigned long long *counters, cudaStream_t st, StepCtl ctl);
cudaError_t launch_wimage(bool cplx, const double *W, int kmax, const int32_t *pairs, int npairs,
                          const int32_t *cexp, const UpdDigits &ud, cudaStream_t st,
                          StepCtl ctl = StepCtl());
size_t ud_scratch_bytes(int nctas, int tmax);
int ud_max_tiles(bool cplx, int kmax);
int ud_num_ctas();
// Digit helpers shared by the inner solve (W-side digits) and the digit kernels.
__device__ __forceinline__ unsigned long long dg_mag_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ int dg_exp_of_bits(unsigned long long mag) {
    const int E = (int)((mag >> 52) & 0x7FF);
    return E == 0 ? -1021 : E - 1022;
}
// floor(|x| 2^(63-e)) for |x| < 2^e (integer shifts of the significand)
__device__ __forceinline__ unsigned long long dg_fixed63(double x, int e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0) return 0ull;
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - 1012 - e;
    if (sh >= 0) return mant << sh;
    if (sh <= -64) return 0ull;
    return mant >> (-sh);
}
// 7-bit digit t (1-based) of two fixed-point values as packed fp16 bits, signed
// by n0, n1. A digit d <= 127 comes out exactly as (1024 + d) - 1024 in fp16:
// the bit pattern of +-(1024 + d) is (0x6400 or 0xE400) | d, and adding -+1024
// leaves +-d. Per pair of digits: two field extracts, a byte permute, an OR and
// one f16x2 add (the sign-dependent constants are loop invariants).
__device__ __forceinline__ uint32_t dg_digits2_bits(unsigned long long q0, bool n0,
                                                    unsigned long long q1, bool n1, int t) {
    const uint32_t bias = (n0 ? 0xE400u : 0x6400u) | ((n1 ? 0xE400u : 0x6400u) << 16);
    const uint32_t add = bias ^ 0x80008000u;  // -1024 for a positive lane, +1024 for a negative one
    const uint32_t d0 = (uint32_t)(q0 >> (63 - 7 * t)) & 127u;
    const uint32_t d1 = (uint32_t)(q1 >> (63 - 7 * t)) & 127u;
    const uint32_t v = __byte_perm(d0, d1, 0x5410) | bias;
    uint32_t r;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(add));
    return r;
}
__device__ __forceinline__ uint32_t dg_sw128_off(int row, int kbyte) {
    return (uint32_t)(row * 128 + ((((kbyte >> 4) ^ (row & 7))) << 4) + (kbyte & 15));
}

// Copy the pivot columns of one pair, rows [l0, l1), from Gs to Gd (pass-through).
__device__ __forceinline__ void pair_copy_rows(bool cplx, const double *Gs, double *Gd, int64_t ld,
                                               const int32_t *pd, int64_t l0, int64_t l1,
                                               int c0, int c1, int tid, int nthreads) {
    const int nc = c1 - c0;
    const int64_t nr = l1 - l0;
    for (int64_t t = tid; t < nr * nc; t += nthreads) {
        const int a = c0 + (int)(t / nr);
        const int64_t l = l0 + t % nr;
        const int64_t col = a < pd[1] ? (int64_t)pd[0] + a : (int64_t)pd[2] + (a - pd[1]);
        if (cplx)
            reinterpret_cast<double2 *>(Gd)[col * ld + l] = reinterpret_cast<const double2 *>(Gs)[col * ld + l];
        else
            Gd[col * ld + l] = Gs[col * ld + l];
    }
}

// Batched solve: problems <-> one work matrix (jj_batch.cu).
cudaError_t launch_batch_gather(bool cplx, const double *const *src, const int64_t *ld,
                                const int64_t *rows, const int32_t *colprob,
                                const int32_t *srccol, double *Gw, int64_t ldw, int64_t ncols,
                                cudaStream_t st);
cudaError_t launch_batch_scatter(bool cplx, const double *Gw, int64_t ldw, double *const *dst,
                                 const int64_t *ld, const int64_t *rows, const int32_t *colprob,
                                 const int32_t *srccol, const int64_t *lamoff, const int8_t *Jw,
                                 double *lambda, int64_t ncols, cudaStream_t st);

// Three-level form: outer Cholesky into the inner work matrix, and the hand-back
// of W_P after the inner sweeps (jj_three.cu).
cudaError_t launch_three_cholesky(bool cplx, const double *A, int kmax, const int32_t *pairs,
                                  int npairs, const int8_t *J, double *X, int64_t ldx, int8_t *JX,
                                  int32_t *fail, unsigned long long *counters, cudaStream_t st,
                                  StepCtl ctl);
cudaError_t launch_three_finish(bool cplx, const double *X, int64_t ldx, int kmax,
                                const int32_t *pairs, int npairs, double *W,
                                const unsigned long long *inner_rot, const int32_t *fail,
                                unsigned long long *counters, cudaStream_t st, StepCtl ctl);

// Front end H -> (G, J) (jj_frontend.cu); returns a jj_status.
int frontend_factor(bool cplx, const double *H, int64_t ldh, int n, double rank_tol, double *G,
                    int64_t ldg, int8_t *J_host, int32_t *perm_host, int8_t *psize_host,
                    int64_t *rank_host, uint64_t wait_ns, cudaStream_t st);

// Host-side ordering tables (jj_schedule.cpp).
int schedule_pairs(int nbl, int order, int sweep, int32_t *pairs);

}  // namespace jj
