// Plain (non-blocked) one-sided J-Jacobi kernels: column norms, the fused
// pair step (dot product, rotation parameters, column update), eigenpair
// extraction and column permutation.
//
// Layout: G column-major, leading dimension ld; complex entries are (re, im)
// double pairs, loaded as one 16-byte double2 per entry (coalesced: a warp
// reads 512 contiguous bytes of a column).
#include "jj_common.cuh"

namespace jj {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of two values over the block (all threads receive the result).
__device__ __forceinline__ void block_sum2(double &a, double &b, double (*sh)[2]) {
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[w][0] = a;
        sh[w][1] = b;
    }
    __syncthreads();
    if (w == 0) {
        a = l < kWarps ? sh[l][0] : 0.0;
        b = l < kWarps ? sh[l][1] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
        if (l == 0) {
            sh[0][0] = a;
            sh[0][1] = b;
        }
    }
    __syncthreads();
    a = sh[0][0];
    b = sh[0][1];
}

// d[c] = ||g_c||^2, one block per column.
template <bool CPLX>
__global__ void __launch_bounds__(kThreads) norms_kernel(const double *__restrict__ G, int64_t ld,
                                                          int64_t m, double *__restrict__ d) {
    __shared__ double sh[kWarps][2];
    const int64_t c = blockIdx.x;
    double acc = 0.0, dummy = 0.0;
    if (CPLX) {
        const double2 *g = reinterpret_cast<const double2 *>(G) + c * ld;
        for (int64_t l = threadIdx.x; l < m; l += kThreads) {
            const double2 v = g[l];
            acc = fma(v.x, v.x, fma(v.y, v.y, acc));
        }
    } else {
        const double *g = G + c * ld;
        for (int64_t l = threadIdx.x; l < m; l += kThreads) acc = fma(g[l], g[l], acc);
    }
    block_sum2(acc, dummy, sh);
    if (threadIdx.x == 0) d[c] = acc;
}

// One parallel step of the plain method: one block per pivot pair (r, s).
// Pass 1 forms a_rs = g_r^* g_s (entries cached in registers, CACHE per
// thread and column); one thread decides and computes the rotation and the
// tracked diagonal; pass 2 rotates the cached entries (and re-reads the rest
// when m exceeds the cache).
template <bool CPLX, int CACHE>
__global__ void __launch_bounds__(kThreads) plain_step_kernel(
    double *__restrict__ G, int64_t ld, int64_t m, int64_t n, const int32_t *__restrict__ pairs,
    const int8_t *__restrict__ J, double *__restrict__ d, double tol,
    unsigned long long *__restrict__ counters) {
    __shared__ double sh[kWarps][2];
    __shared__ Rot rot;
    __shared__ int apply;
    int r = pairs[2 * blockIdx.x], s = pairs[2 * blockIdx.x + 1];
    if (r >= n || s >= n || r < 0 || s < 0) return;  // dummy column of an odd order
    if (r > s) {
        const int t = r;
        r = s;
        s = t;
    }
    const int tid = threadIdx.x;
    double sr = 0.0, si = 0.0;
    if (CPLX) {
        double2 *gr = reinterpret_cast<double2 *>(G) + (int64_t)r * ld;
        double2 *gs = reinterpret_cast<double2 *>(G) + (int64_t)s * ld;
        double2 x[CACHE], y[CACHE];
#pragma unroll
        for (int k = 0; k < CACHE; ++k) {
            const int64_t l = tid + (int64_t)k * kThreads;
            if (l < m) {
                x[k] = gr[l];
                y[k] = gs[l];
                sr = fma(x[k].x, y[k].x, fma(x[k].y, y[k].y, sr));
                si = fma(x[k].x, y[k].y, fma(-x[k].y, y[k].x, si));
            }
        }
        for (int64_t l = tid + (int64_t)CACHE * kThreads; l < m; l += kThreads) {
            const double2 a = gr[l], b = gs[l];
            sr = fma(a.x, b.x, fma(a.y, b.y, sr));
            si = fma(a.x, b.y, fma(-a.y, b.x, si));
        }
        block_sum2(sr, si, sh);
        if (tid == 0) {
            const double dr = d[r], ds = d[s];
            const double absa = sqrt(sr * sr + si * si);
            const double rel = absa / sqrt(dr * ds);
            int ap = 0;
            if (!isfinite(rel)) {
                atomicOr(&counters[kCntErr], kErrNonfinite);
            } else {
                atomic_max_nonneg(&counters[kCntMaxOff], rel);
                if (rel > tol) {
                    Rot R;
                    if (rotation(dr, ds, sr, si, (int)J[r] * (int)J[s], true, R)) {
                        rot = R;
                        d[r] = R.dr;
                        d[s] = R.ds;
                        ap = 1;
                        atomicAdd(&counters[kCntRot], 1ull);
                    } else {
                        atomicOr(&counters[kCntErr], kErrNotPosdef);
                    }
                }
            }
            apply = ap;
        }
        __syncthreads();
        if (!apply) return;
        const Rot R = rot;
#pragma unroll
        for (int k = 0; k < CACHE; ++k) {
            const int64_t l = tid + (int64_t)k * kThreads;
            if (l < m) {
                rot_apply_c(R, x[k].x, x[k].y, y[k].x, y[k].y);
                gr[l] = x[k];
                gs[l] = y[k];
            }
        }
        for (int64_t l = tid + (int64_t)CACHE * kThreads; l < m; l += kThreads) {
            double2 a = gr[l], b = gs[l];
            rot_apply_c(R, a.x, a.y, b.x, b.y);
            gr[l] = a;
            gs[l] = b;
        }
    } else {
        double *gr = G + (int64_t)r * ld;
        double *gs = G + (int64_t)s * ld;
        double x[CACHE], y[CACHE];
#pragma unroll
        for (int k = 0; k < CACHE; ++k) {
            const int64_t l = tid + (int64_t)k * kThreads;
            if (l < m) {
                x[k] = gr[l];
                y[k] = gs[l];
                sr = fma(x[k], y[k], sr);
            }
        }
        for (int64_t l = tid + (int64_t)CACHE * kThreads; l < m; l += kThreads)
            sr = fma(gr[l], gs[l], sr);
        block_sum2(sr, si, sh);
        if (tid == 0) {
            const double dr = d[r], ds = d[s];
            const double rel = fabs(sr) / sqrt(dr * ds);
            int ap = 0;
            if (!isfinite(rel)) {
                atomicOr(&counters[kCntErr], kErrNonfinite);
            } else {
                atomic_max_nonneg(&counters[kCntMaxOff], rel);
                if (rel > tol) {
                    Rot R;
                    if (rotation(dr, ds, sr, 0.0, (int)J[r] * (int)J[s], false, R)) {
                        rot = R;
                        d[r] = R.dr;
                        d[s] = R.ds;
                        ap = 1;
                        atomicAdd(&counters[kCntRot], 1ull);
                    } else {
                        atomicOr(&counters[kCntErr], kErrNotPosdef);
                    }
                }
            }
            apply = ap;
        }
        __syncthreads();
        if (!apply) return;
        const Rot R = rot;
#pragma unroll
        for (int k = 0; k < CACHE; ++k) {
            const int64_t l = tid + (int64_t)k * kThreads;
            if (l < m) {
                rot_apply_r(R, x[k], y[k]);
                gr[l] = x[k];
                gs[l] = y[k];
            }
        }
        for (int64_t l = tid + (int64_t)CACHE * kThreads; l < m; l += kThreads) {
            double a = gr[l], b = gs[l];
            rot_apply_r(R, a, b);
            gr[l] = a;
            gs[l] = b;
        }
    }
}

// lambda[out] = J[c] ||g_c||^2 and u_out = g_c / ||g_c|| (out = perm[c] or c).
template <bool CPLX>
__global__ void __launch_bounds__(kThreads) extract_kernel(
    const double *__restrict__ G, int64_t ld, int64_t m, const int8_t *__restrict__ J,
    const int32_t *__restrict__ perm, double *__restrict__ lambda, double *__restrict__ U,
    int64_t ldu) {
    __shared__ double sh[kWarps][2];
    const int64_t c = blockIdx.x;
    const int64_t o = perm ? perm[c] : c;
    double acc = 0.0, dummy = 0.0;
    if (CPLX) {
        const double2 *g = reinterpret_cast<const double2 *>(G) + c * ld;
        for (int64_t l = threadIdx.x; l < m; l += kThreads) {
            const double2 v = g[l];
            acc = fma(v.x, v.x, fma(v.y, v.y, acc));
        }
    } else {
        const double *g = G + c * ld;
        for (int64_t l = threadIdx.x; l < m; l += kThreads) acc = fma(g[l], g[l], acc);
    }
    block_sum2(acc, dummy, sh);
    if (threadIdx.x == 0) lambda[o] = (double)J[c] * acc;
    if (U) {
        const double inv = 1.0 / sqrt(acc);
        if (CPLX) {
            const double2 *g = reinterpret_cast<const double2 *>(G) + c * ld;
            double2 *u = reinterpret_cast<double2 *>(U) + o * ldu;
            for (int64_t l = threadIdx.x; l < m; l += kThreads) {
                const double2 v = g[l];
                u[l] = make_double2(v.x * inv, v.y * inv);
            }
        } else {
            const double *g = G + c * ld;
            double *u = U + o * ldu;
            for (int64_t l = threadIdx.x; l < m; l += kThreads) u[l] = g[l] * inv;
        }
    }
}

template <bool CPLX>
__global__ void __launch_bounds__(kThreads) permute_kernel(const double *__restrict__ A,
                                                            int64_t lda, double *__restrict__ B,
                                                            int64_t ldb, int64_t m,
                                                            const int32_t *__restrict__ perm,
                                                            int scatter) {
    const int64_t c = blockIdx.x;
    const int64_t src = scatter ? c : perm[c];
    const int64_t dst = scatter ? perm[c] : c;
    if (CPLX) {
        const double2 *a = reinterpret_cast<const double2 *>(A) + src * lda;
        double2 *b = reinterpret_cast<double2 *>(B) + dst * ldb;
        for (int64_t l = threadIdx.x; l < m; l += kThreads) b[l] = a[l];
    } else {
        const double *a = A + src * lda;
        double *b = B + dst * ldb;
        for (int64_t l = threadIdx.x; l < m; l += kThreads) b[l] = a[l];
    }
}

}  // namespace

cudaError_t launch_column_norms(bool cplx, const double *G, int64_t ld, int64_t m, int64_t n,
                                double *d, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (cplx)
        norms_kernel<true><<<(unsigned)n, kThreads, 0, st>>>(G, ld, m, d);
    else
        norms_kernel<false><<<(unsigned)n, kThreads, 0, st>>>(G, ld, m, d);
    return cudaGetLastError();
}

cudaError_t launch_plain_step(bool cplx, double *G, int64_t ld, int64_t m, int64_t n,
                              const int32_t *pairs, int npairs, const int8_t *J, double *d,
                              double tol, unsigned long long *counters, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    // Entries per thread kept in registers between the two passes.
    if (cplx) {
        if (m <= 2 * kThreads)
            plain_step_kernel<true, 2><<<npairs, kThreads, 0, st>>>(G, ld, m, n, pairs, J, d, tol, counters);
        else
            plain_step_kernel<true, 8><<<npairs, kThreads, 0, st>>>(G, ld, m, n, pairs, J, d, tol, counters);
    } else {
        if (m <= 2 * kThreads)
            plain_step_kernel<false, 2><<<npairs, kThreads, 0, st>>>(G, ld, m, n, pairs, J, d, tol, counters);
        else
            plain_step_kernel<false, 16><<<npairs, kThreads, 0, st>>>(G, ld, m, n, pairs, J, d, tol, counters);
    }
    return cudaGetLastError();
}

cudaError_t launch_extract(bool cplx, const double *G, int64_t ld, int64_t m, int64_t n,
                           const int8_t *J, const int32_t *perm, double *lambda, double *U,
                           int64_t ldu, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (cplx)
        extract_kernel<true><<<(unsigned)n, kThreads, 0, st>>>(G, ld, m, J, perm, lambda, U, ldu);
    else
        extract_kernel<false><<<(unsigned)n, kThreads, 0, st>>>(G, ld, m, J, perm, lambda, U, ldu);
    return cudaGetLastError();
}

cudaError_t launch_permute_columns(bool cplx, const double *A, int64_t lda, double *B,
                                   int64_t ldb, int64_t m, int64_t n, const int32_t *perm,
                                   bool scatter, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (cplx)
        permute_kernel<true><<<(unsigned)n, kThreads, 0, st>>>(A, lda, B, ldb, m, perm, scatter);
    else
        permute_kernel<false><<<(unsigned)n, kThreads, 0, st>>>(A, lda, B, ldb, m, perm, scatter);
    return cudaGetLastError();
}

}  // namespace jj
