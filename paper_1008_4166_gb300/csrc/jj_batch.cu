// Batched solve: moving many independent problems of uneven order into one
// work matrix and back. Problem p occupies the work columns
// [coff_p, coff_p + n_p), in J-sorted order, rows [0, m_p); the rows below m_p
// (up to the common leading dimension) are zero and stay zero, because every
// kernel of the sweep works only on the rows of the pair's own problem.
#include "jj_common.cuh"

namespace jj {
namespace {

constexpr int kThreads = 256;

// Work column c <- column srccol[c] of problem colprob[c]; rows m_p.. zeroed.
template <bool CPLX>
__global__ void __launch_bounds__(kThreads) batch_gather_kernel(
    const double *const *__restrict__ src, const int64_t *__restrict__ ld,
    const int64_t *__restrict__ rows, const int32_t *__restrict__ colprob,
    const int32_t *__restrict__ srccol, double *__restrict__ Gw, int64_t ldw) {
    constexpr int E = CPLX ? 2 : 1;
    const int64_t c = blockIdx.x;
    const int p = colprob[c];
    const double *s = src[p] + (int64_t)srccol[c] * ld[p] * E;
    double *d = Gw + c * ldw * E;
    const int64_t mp = rows[p] * E;
    for (int64_t i = threadIdx.x; i < ldw * E; i += kThreads) d[i] = i < mp ? s[i] : 0.0;
}

// Column srccol[c] of problem colprob[c] <- work column c, and
// lambda[lamoff[p] + srccol[c]] = J_cc ||g~_c||^2 (Alg. 5.2, end), with the
// squares summed in the order of the single-problem extraction (per row, rows
// strided over the block, warp then block reduction), so that both give the
// same bits.
template <bool CPLX>
__global__ void __launch_bounds__(kThreads) batch_scatter_kernel(
    const double *__restrict__ Gw, int64_t ldw, double *const *__restrict__ dst,
    const int64_t *__restrict__ ld, const int64_t *__restrict__ rows,
    const int32_t *__restrict__ colprob, const int32_t *__restrict__ srccol,
    const int64_t *__restrict__ lamoff, const int8_t *__restrict__ Jw, double *__restrict__ lambda) {
    __shared__ double sh[kThreads / 32];
    const int64_t c = blockIdx.x;
    const int p = colprob[c];
    const int64_t mp = rows[p];
    double acc = 0.0;
    if (CPLX) {
        const double2 *s = reinterpret_cast<const double2 *>(Gw) + c * ldw;
        double2 *d = reinterpret_cast<double2 *>(dst[p]) + (int64_t)srccol[c] * ld[p];
        for (int64_t l = threadIdx.x; l < mp; l += kThreads) {
            const double2 v = s[l];
            d[l] = v;
            acc = fma(v.x, v.x, fma(v.y, v.y, acc));
        }
    } else {
        const double *s = Gw + c * ldw;
        double *d = dst[p] + (int64_t)srccol[c] * ld[p];
        for (int64_t l = threadIdx.x; l < mp; l += kThreads) {
            const double v = s[l];
            d[l] = v;
            acc = fma(v, v, acc);
        }
    }
    auto warp_sum = [](double v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    acc = warp_sum(acc);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = acc;
    __syncthreads();
    if (w == 0) {
        acc = warp_sum(l < kThreads / 32 ? sh[l] : 0.0);
        if (l == 0 && lambda) lambda[lamoff[p] + srccol[c]] = (double)Jw[c] * acc;
    }
}

}  // namespace

cudaError_t launch_batch_gather(bool cplx, const double *const *src, const int64_t *ld,
                                const int64_t *rows, const int32_t *colprob,
                                const int32_t *srccol, double *Gw, int64_t ldw, int64_t ncols,
                                cudaStream_t st) {
    if (ncols <= 0) return cudaSuccess;
    if (cplx)
        batch_gather_kernel<true><<<(unsigned)ncols, kThreads, 0, st>>>(src, ld, rows, colprob,
                                                                         srccol, Gw, ldw);
    else
        batch_gather_kernel<false><<<(unsigned)ncols, kThreads, 0, st>>>(src, ld, rows, colprob,
                                                                          srccol, Gw, ldw);
    return cudaGetLastError();
}

cudaError_t launch_batch_scatter(bool cplx, const double *Gw, int64_t ldw, double *const *dst,
                                 const int64_t *ld, const int64_t *rows, const int32_t *colprob,
                                 const int32_t *srccol, const int64_t *lamoff, const int8_t *Jw,
                                 double *lambda, int64_t ncols, cudaStream_t st) {
    if (ncols <= 0) return cudaSuccess;
    if (cplx)
        batch_scatter_kernel<true><<<(unsigned)ncols, kThreads, 0, st>>>(
            Gw, ldw, dst, ld, rows, colprob, srccol, lamoff, Jw, lambda);
    else
        batch_scatter_kernel<false><<<(unsigned)ncols, kThreads, 0, st>>>(
            Gw, ldw, dst, ld, rows, colprob, srccol, lamoff, Jw, lambda);
    return cudaGetLastError();
}

}  // namespace jj
