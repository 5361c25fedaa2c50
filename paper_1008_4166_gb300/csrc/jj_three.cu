// Three-level forms (Sec. 5.1-5.2, cases 3F and 3B): the inner J-Jacobi of
// every outer pivot pair is itself the blocked method (Alg. 3.3 on R; for 3B
// one block-oriented pass, over every inner block pair in the first outer step
// of a sweep and over the cross pairs of Alg. 5.1 in the others). Outer pair q owns
// the slice X_q = [R_q; W_q] of an inner work matrix (columns
// [q kmax, q kmax + k_q), leading dimension ldx >= 2 kmax): R_q (rows
// [0, kmax)) is the Cholesky factor of the outer Gram block (3.8) and W_q
// (rows [kmax, 2 kmax)) starts as I. The one-sided inner method forms its
// Gram blocks from the R rows only and applies every inner transformation to
// both parts, so that at the end R_q W_q and W_q = the accumulated transform
// (3.12) sit in X_q. The inner steps run the ordinary Gram, inner-pivot and
// update kernels over all outer pairs at once; this file holds the two kernels
// around them.
#include "jj_common.cuh"

namespace jj {
namespace {

constexpr int CT = 512;  // threads per block

__device__ __forceinline__ int64_t piv_col(const int32_t *pd, int a) {
    return a < pd[1] ? (int64_t)pd[0] + a : (int64_t)pd[2] + (a - pd[1]);
}

// Set X_q to [I; I] (an inner problem with nothing to do).
template <bool CPLX>
__device__ void x_identity(double *Xq, int64_t ldx, int kmax, int k) {
    constexpr int E = CPLX ? 2 : 1;
    for (int64_t t = threadIdx.x; t < (int64_t)kmax * 2 * kmax; t += CT) {
        const int b = (int)(t / (2 * kmax)), r = (int)(t % (2 * kmax));
        const int a = r < kmax ? r : r - kmax;
        double *x = Xq + ((int64_t)b * ldx + r) * E;
        x[0] = (a == b && b < k) ? 1.0 : 0.0;
        if (CPLX) x[1] = 0.0;
    }
}

// One block per outer pair: the upper Cholesky factor of A_P (right-looking,
// in place in the R rows of X_q, which stay in L2), W_q = I, and J of the
// pivot columns into JX. Skipped outer pairs get X_q = [I; I] (the inner
// method then finds nothing to rotate); a failed factorisation (A_P not
// positive definite in working precision) is flagged and gets [I; I] too.
template <bool CPLX>
__global__ void __launch_bounds__(CT) three_cholesky_kernel(
    const double *__restrict__ A, int kmax, const int32_t *__restrict__ pairs,
    const int8_t *__restrict__ J, double *__restrict__ X, int64_t ldx, int8_t *__restrict__ JX,
    int32_t *__restrict__ fail, unsigned long long *__restrict__ counters, StepCtl ctl) {
    constexpr int E = CPLX ? 2 : 1;
    __shared__ int s_fail;
    __shared__ double s_piv;
    const int q = blockIdx.x, tid = threadIdx.x;
    const int32_t *pd = pairs + 4 * q;
    const int k = pd[1] + pd[3];
    double *Xq = X + (int64_t)q * kmax * ldx * E;
    for (int a = tid; a < kmax; a += CT) JX[(int64_t)q * kmax + a] = a < k ? J[piv_col(pd, a)] : (int8_t)1;
    if (tid == 0) fail[q] = 0;
    if (ctl.flags && (ctl.flags[q] & kPairSkipped)) {
        x_identity<CPLX>(Xq, ldx, kmax, k);
        return;
    }
    const double *Aq = A + (int64_t)q * kmax * kmax * E;
    // R rows: upper triangle of A_P, zero elsewhere; W rows: I
    for (int64_t t = tid; t < (int64_t)kmax * 2 * kmax; t += CT) {
        const int b = (int)(t / (2 * kmax)), r = (int)(t % (2 * kmax));
        double *x = Xq + ((int64_t)b * ldx + r) * E;
        if (r < kmax) {
            const bool in = r <= b && b < k;
#pragma unroll
            for (int e = 0; e < E; ++e) x[e] = in ? Aq[((int64_t)b * kmax + r) * E + e] : 0.0;
        } else {
            x[0] = (r - kmax == b && b < k) ? 1.0 : 0.0;
            if (CPLX) x[1] = 0.0;
        }
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    auto R = [&](int r, int c) -> double * { return Xq + ((int64_t)c * ldx + r) * E; };
    for (int j = 0; j < k; ++j) {
        if (tid == 0) {
            const double ajj = R(j, j)[0];
            if (!(ajj > 0.0) || !isfinite(ajj)) {
                s_fail = 1;
                s_piv = 1.0;
            } else {
                s_piv = sqrt(ajj);
            }
        }
        __syncthreads();
        if (s_fail) break;
        const double rjj = s_piv, inv = 1.0 / rjj;
        for (int l = j + 1 + tid; l < k; l += CT) {
#pragma unroll
            for (int e = 0; e < E; ++e) R(j, l)[e] *= inv;
        }
        if (tid == 0) {
            R(j, j)[0] = rjj;
            if (CPLX) R(j, j)[1] = 0.0;
        }
        __syncthreads();
        const int rem = k - j - 1;
        for (int t = tid; t < rem * rem; t += CT) {
            const int c1 = j + 1 + t % rem, c2 = j + 1 + t / rem;
            if (c1 > c2) continue;
            if (CPLX) {
                const double ur = R(j, c1)[0], ui = R(j, c1)[1];
                const double vr = R(j, c2)[0], vi = R(j, c2)[1];
                double *dst = R(c1, c2);
                dst[0] -= fma(ur, vr, ui * vi);
                dst[1] -= fma(ur, vi, -ui * vr);
            } else {
                R(c1, c2)[0] -= R(j, c1)[0] * R(j, c2)[0];
            }
        }
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) {
            fail[q] = 1;
            atomicOr(&counters[kCntErr], kErrNotPosdef);
        }
        __syncthreads();
        x_identity<CPLX>(Xq, ldx, kmax, k);
    }
}

// One block per outer pair, after the inner sweeps: W_P (the W rows of X_q)
// into the pivot block array for the outer update, and the outer pair's
// bookkeeping (rotations applied by its inner solve, skip stamps, errors).
template <bool CPLX>
__global__ void __launch_bounds__(CT) three_finish_kernel(
    const double *__restrict__ X, int64_t ldx, int kmax, const int32_t *__restrict__ pairs,
    double *__restrict__ Wb, const unsigned long long *__restrict__ inner_rot,
    const int32_t *__restrict__ fail, unsigned long long *__restrict__ counters, StepCtl ctl) {
    constexpr int E = CPLX ? 2 : 1;
    const int q = blockIdx.x, tid = threadIdx.x;
    const int32_t *pd = pairs + 4 * q;
    if (ctl.flags && (ctl.flags[q] & kPairSkipped)) return;
    const int k = pd[1] + pd[3];
    const double *Xq = X + (int64_t)q * kmax * ldx * E;
    double *Wq = Wb + (int64_t)q * kmax * kmax * E;
    for (int t = tid; t < k * k; t += CT) {
        const int a = t % k, b = t / k;
#pragma unroll
        for (int e = 0; e < E; ++e) Wq[((int64_t)b * kmax + a) * E + e] = Xq[((int64_t)b * ldx + kmax + a) * E + e];
    }
    if (tid == 0) {
        const unsigned long long rot = inner_rot[2 * q];
        const unsigned long long err = inner_rot[2 * q + 1];
        const bool failed = fail[q] != 0 || err != 0;
        if (err) atomicOr(&counters[kCntErr], err);
        if (rot) atomicAdd(&counters[kCntRot], rot);
        atomicAdd(&counters[kCntPairs], 1ull);
        if (rot) atomicAdd(&counters[kCntPairsRot], 1ull);
        pair_record(ctl, pd, q, rot > 0 && !failed, failed);
        pair_count_prob(ctl, q, rot);
        if (err) pair_flag_prob(ctl, q, err);
    }
}

}  // namespace

cudaError_t launch_three_cholesky(bool cplx, const double *A, int kmax, const int32_t *pairs,
                                  int npairs, const int8_t *J, double *X, int64_t ldx, int8_t *JX,
                                  int32_t *fail, unsigned long long *counters, cudaStream_t st,
                                  StepCtl ctl) {
    if (npairs <= 0) return cudaSuccess;
    if (cplx)
        three_cholesky_kernel<true><<<npairs, CT, 0, st>>>(A, kmax, pairs, J, X, ldx, JX, fail,
                                                           counters, ctl);
    else
        three_cholesky_kernel<false><<<npairs, CT, 0, st>>>(A, kmax, pairs, J, X, ldx, JX, fail,
                                                            counters, ctl);
    return cudaGetLastError();
}

cudaError_t launch_three_finish(bool cplx, const double *X, int64_t ldx, int kmax,
                                const int32_t *pairs, int npairs, double *W,
                                const unsigned long long *inner_rot, const int32_t *fail,
                                unsigned long long *counters, cudaStream_t st, StepCtl ctl) {
    if (npairs <= 0) return cudaSuccess;
    if (cplx)
        three_finish_kernel<true><<<npairs, CT, 0, st>>>(X, ldx, kmax, pairs, W, inner_rot, fail,
                                                         counters, ctl);
    else
        three_finish_kernel<false><<<npairs, CT, 0, st>>>(X, ldx, kmax, pairs, W, inner_rot, fail,
                                                          counters, ctl);
    return cudaGetLastError();
}

}  // namespace jj
