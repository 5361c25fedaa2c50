// Front end of the method: the Hermitian indefinite factorization
// H -> (G, J) with H = G J G^* of Sec. 2.2, (2.5).
//
// Symmetric Gaussian elimination with complete (Bunch-Parlett) pivoting,
// P H P^T = M D M^*: at every step, mu0 is the largest modulus of the Schur
// complement S and mu1 the largest modulus on its diagonal; a 1x1 pivot at
// the largest diagonal entry when mu1 >= alpha mu0 (alpha = (1 + sqrt 17)/8),
// else the 2x2 pivot on the off-diagonal entry of modulus mu0. Ties go to the
// first entry in row-major order of S. Elimination stops when mu0 falls to
// rank_tol times the largest modulus of H (rank r). The columns of M are then
// scaled by the blocks of D: a 1x1 block d gives the column M_k |d|^(1/2) with
// sign(d); a 2x2 block E = Q diag(delta) Q^* gives M_b Q |delta|^(1/2) with
// signs sign(delta). The rows of G are returned to H's order.
//
// One cooperative kernel over every SM runs the elimination; each step has
// one grid barrier after each interchange and one after the update (bounded
// waits: a barrier that runs out sets an error flag and every block returns):
//   1. every block reduces the block-local maxima left by the previous update
//      to the same pivot decision; the symmetric interchanges follow, one
//      pass each;
//   2. every block updates its share of the trailing lower triangle,
//      T = S - L C^* with L = C E^{-1} (rank 1 or 2), with a real diagonal,
//      writes the rows of M, and records the maxima of its share for the next
//      step.
// Only the lower triangle of the Hermitian matrix is stored and read (in a
// column-major workspace), so S stays exactly Hermitian by construction.
#include <cuda_runtime.h>

#include <vector>

#include "jj_common.cuh"
#include "jj_tc.cuh"

namespace jj {
namespace {

constexpr int FE_THREADS = 256;
constexpr double kAlphaBP = 0.64038820320220756;  // (1 + sqrt(17)) / 8

struct FeMax {
    double mu0;        // largest modulus off the diagonal
    long long key0;    // i * n + j of its upper copy (i < j): row-major position
    double mu1;        // largest modulus on the diagonal
    long long key1;    // its index
};

struct FeState {
    unsigned int count;  // grid barrier arrivals
    unsigned int gen;    // grid barrier generation
    int err;             // 1: a barrier wait ran out
    int rank;
    double mu0_init;
};

template <bool CPLX>
struct Cx {
    double re, im;
};

__device__ __forceinline__ bool fe_better(double v, long long key, double bv, long long bkey) {
    return v > bv || (v == bv && key < bkey);
}

// Bounded grid barrier (all blocks resident: cooperative launch). Memory
// written before it is visible to every block after it.
__device__ bool fe_grid_sync(FeState *st, unsigned int nblocks, uint64_t limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int *vgen = &st->gen;
        const unsigned int g = *vgen;
        __threadfence();
        if (atomicAdd(&st->count, 1u) == nblocks - 1) {
            st->count = 0;
            __threadfence();
            atomicAdd(&st->gen, 1u);
        } else {
            const uint64_t t0 = tc::global_ns();
            long it = 0;
            while (*vgen == g) {
                if (((++it) & 63) == 0 && (tc::global_ns() - t0 > limit_ns || *(volatile int *)&st->err)) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (!ok) atomicExch(&st->err, 1);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <bool CPLX>
__device__ __forceinline__ double fe_abs(const double *A, int64_t idx) {
    if (CPLX) return hypot(A[2 * idx], A[2 * idx + 1]);
    return fabs(A[idx]);
}

// Elimination: A (n x n, ld n, full Hermitian, overwritten), M (n x n, ld n,
// columns 0..r-1 written), perm (n), psize (n: 1 or 2 at the first column of
// each pivot, 0 at the second), state, per-block maxima (2 x nblocks, double
// buffered by step parity).
template <bool CPLX>
__global__ void __launch_bounds__(FE_THREADS) fe_eliminate_kernel(
    double *__restrict__ A, double *__restrict__ M, int n, int32_t *__restrict__ perm,
    int8_t *__restrict__ psize, FeState *st, FeMax *__restrict__ bmax, double rank_tol,
    uint64_t wait_ns) {
    constexpr int E = CPLX ? 2 : 1;
    const unsigned int nb = gridDim.x;
    const long long gtid = (long long)blockIdx.x * FE_THREADS + threadIdx.x;
    const long long gthreads = (long long)nb * FE_THREADS;
    __shared__ FeMax s_red[FE_THREADS / 32];
    __shared__ int s_piv[2], s_s, s_stop;
    __shared__ double s_einv[8];  // E^{-1} (s x s, complex interleaved, column-major)

    auto at = [&](int i, int j) -> int64_t { return (int64_t)j * n + i; };

    // block-local maxima (off the diagonal and on it) of the entries each
    // thread visited, written to bmax[par * nb + block]
    auto block_max = [&](FeMax mine, int par) {
        // warp reduction, then block
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v0 = __shfl_down_sync(0xffffffffu, mine.mu0, o);
            const long long k0 = __shfl_down_sync(0xffffffffu, mine.key0, o);
            const double v1 = __shfl_down_sync(0xffffffffu, mine.mu1, o);
            const long long k1 = __shfl_down_sync(0xffffffffu, mine.key1, o);
            if (fe_better(v0, k0, mine.mu0, mine.key0)) {
                mine.mu0 = v0;
                mine.key0 = k0;
            }
            if (fe_better(v1, k1, mine.mu1, mine.key1)) {
                mine.mu1 = v1;
                mine.key1 = k1;
            }
        }
        if (lane == 0) s_red[warp] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            FeMax b = s_red[0];
            for (int w = 1; w < FE_THREADS / 32; ++w) {
                if (fe_better(s_red[w].mu0, s_red[w].key0, b.mu0, b.key0)) {
                    b.mu0 = s_red[w].mu0;
                    b.key0 = s_red[w].key0;
                }
                if (fe_better(s_red[w].mu1, s_red[w].key1, b.mu1, b.key1)) {
                    b.mu1 = s_red[w].mu1;
                    b.key1 = s_red[w].key1;
                }
            }
            bmax[par * nb + blockIdx.x] = b;
        }
        __syncthreads();
    };

    // maxima of the whole matrix (step 0)
    {
        FeMax mine{-1.0, 0x7fffffffffffffffll, -1.0, 0x7fffffffffffffffll};
        const long long tot = (long long)n * n;
        for (long long t = gtid; t < tot; t += gthreads) {
            const int i = (int)(t % n), j = (int)(t / n);
            if (i < j) continue;
            const double v = fe_abs<CPLX>(A, at(i, j));
            if (i == j) {
                if (fe_better(v, i, mine.mu1, mine.key1)) {
                    mine.mu1 = v;
                    mine.key1 = i;
                }
            } else if (fe_better(v, (long long)j * n + i, mine.mu0, mine.key0)) {
                mine.mu0 = v;  // key: the row-major position of the upper copy (j, i)
                mine.key0 = (long long)j * n + i;
            }
        }
        block_max(mine, 0);
    }
    if (!fe_grid_sync(st, nb, wait_ns)) return;

    double mu0_init = -1.0;
    int k = 0, par = 0;
    while (k < n) {
        // ---- 1. pivot decision (the same in every block) ----
        if (threadIdx.x == 0) {
            FeMax b{-1.0, 0x7fffffffffffffffll, -1.0, 0x7fffffffffffffffll};
            for (unsigned int q = 0; q < nb; ++q) {
                const FeMax c = bmax[par * nb + q];
                if (fe_better(c.mu0, c.key0, b.mu0, b.key0)) {
                    b.mu0 = c.mu0;
                    b.key0 = c.key0;
                }
                if (fe_better(c.mu1, c.key1, b.mu1, b.key1)) {
                    b.mu1 = c.mu1;
                    b.key1 = c.key1;
                }
            }
            const double mu0 = fmax(b.mu0, b.mu1);  // largest modulus of S
            if (k == 0) mu0_init = mu0;
            s_stop = (mu0 <= 0.0 || mu0 <= rank_tol * mu0_init) ? 1 : 0;
            if (b.mu1 >= kAlphaBP * mu0 || k == n - 1 || b.mu0 < 0.0) {
                s_s = 1;
                s_piv[0] = (int)b.key1;
            } else {
                s_s = 2;
                s_piv[0] = (int)(b.key0 / n);  // i < j
                s_piv[1] = (int)(b.key0 % n);
            }
        }
        __syncthreads();
        if (s_stop) break;
        const int s = s_s;
        // symmetric interchanges: pivot t to position k + t (piv[0] < piv[1], so
        // the first interchange never moves the second pivot). Only the lower
        // triangle of S is stored; swapping rows and columns d < p of a
        // Hermitian matrix moves each stored entry to a stored position, the
        // entries between d and p crossing the diagonal (conjugated). Thread x
        // owns the entries of index x, so one pass has no conflicts.
        for (int t = 0; t < s; ++t) {
            const int p = s_piv[t], d = k + t;
            if (p == d) continue;
            for (long long xx = gtid; xx < n; xx += gthreads) {
                const int x = (int)xx;
                if (x < k) {  // the computed columns of M: rows d and p
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const double y = M[at(d, x) * E + e];
                        M[at(d, x) * E + e] = M[at(p, x) * E + e];
                        M[at(p, x) * E + e] = y;
                    }
                } else if (x < d) {  // S(d, x) <-> S(p, x)
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const double y = A[at(d, x) * E + e];
                        A[at(d, x) * E + e] = A[at(p, x) * E + e];
                        A[at(p, x) * E + e] = y;
                    }
                } else if (x == d) {  // the two diagonal entries; S(p, d) conjugated
                    const double y = A[at(d, d) * E];
                    A[at(d, d) * E] = A[at(p, p) * E];
                    A[at(p, p) * E] = y;
                    if (CPLX) A[at(p, d) * E + 1] = -A[at(p, d) * E + 1];
                } else if (x < p) {  // S(x, d) <-> conj S(p, x)
                    const double yr = A[at(x, d) * E];
                    A[at(x, d) * E] = A[at(p, x) * E];
                    A[at(p, x) * E] = yr;
                    if (CPLX) {
                        const double yi = A[at(x, d) * E + 1];
                        A[at(x, d) * E + 1] = -A[at(p, x) * E + 1];
                        A[at(p, x) * E + 1] = -yi;
                    }
                } else if (x > p) {  // S(x, d) <-> S(x, p)
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const double y = A[at(x, d) * E + e];
                        A[at(x, d) * E + e] = A[at(x, p) * E + e];
                        A[at(x, p) * E + e] = y;
                    }
                }
            }
            if (gtid == 0) {
                const int y = perm[d];
                perm[d] = perm[p];
                perm[p] = y;
            }
            if (!fe_grid_sync(st, nb, wait_ns)) return;
        }
        // ---- 2. E^{-1} (every block), L = C E^{-1}, T = S - L C^* ----
        if (threadIdx.x == 0) {
            if (s == 1) {
                s_einv[0] = 1.0 / A[at(k, k) * E];
                s_einv[1] = 0.0;
            } else {
                // E = [[a, b^*], [b, d]] (a, d real); E^{-1} = [[d, -b^*], [-b, a]] / (a d - |b|^2)
                const double a = A[at(k, k) * E], dd = A[at(k + 1, k + 1) * E];
                const double br = A[at(k + 1, k) * E], bi = CPLX ? A[at(k + 1, k) * E + 1] : 0.0;
                const double det = a * dd - (br * br + bi * bi);
                const double id = 1.0 / det;
                // column-major: (0,0), (1,0), (0,1), (1,1)
                s_einv[0] = dd * id;
                s_einv[1] = 0.0;
                s_einv[2] = -br * id;
                s_einv[3] = -bi * id;
                s_einv[4] = -br * id;
                s_einv[5] = bi * id;
                s_einv[6] = a * id;
                s_einv[7] = 0.0;
            }
        }
        __syncthreads();
        const int k1 = k + s, nt = n - k1;
        // L_i = C_i E^{-1} (row vector), C_i = A[i, k..k+s-1]
        auto lrow = [&](int i, double (&L)[2][2]) {
            double c[2][2];
            for (int t = 0; t < 2; ++t) {
                c[t][0] = t < s ? A[at(i, k + t) * E] : 0.0;
                c[t][1] = (t < s && CPLX) ? A[at(i, k + t) * E + 1] : 0.0;
            }
            for (int u = 0; u < 2; ++u) {
                double lr = 0.0, li = 0.0;
                for (int t = 0; t < s && u < s; ++t) {
                    const double er = s_einv[(u * 2 + t) * 2], ei = s_einv[(u * 2 + t) * 2 + 1];
                    lr += c[t][0] * er - c[t][1] * ei;
                    li += c[t][0] * ei + c[t][1] * er;
                }
                L[u][0] = lr;
                L[u][1] = li;
            }
        };
        FeMax mine{-1.0, 0x7fffffffffffffffll, -1.0, 0x7fffffffffffffffll};
        const long long tot = (long long)nt * nt;
        for (long long t = gtid; t < tot; t += gthreads) {
            const int ii = (int)(t % nt), jj = (int)(t / nt);
            if (ii < jj) continue;  // the stored lower triangle (i >= j)
            const int i = k1 + ii, j = k1 + jj;
            double Li[2][2];
            lrow(i, Li);
            // T_ij = A_ij - sum_t L_it conj(C_jt)
            double tr = A[at(i, j) * E], ti = CPLX ? A[at(i, j) * E + 1] : 0.0;
            for (int u = 0; u < s; ++u) {
                const double cr = A[at(j, k + u) * E], ci = CPLX ? A[at(j, k + u) * E + 1] : 0.0;
                tr -= Li[u][0] * cr + Li[u][1] * ci;
                ti -= Li[u][1] * cr - Li[u][0] * ci;
            }
            if (i == j) {
                A[at(i, i) * E] = tr;
                if (CPLX) A[at(i, i) * E + 1] = 0.0;
                const double v = fabs(tr);
                if (fe_better(v, i, mine.mu1, mine.key1)) {
                    mine.mu1 = v;
                    mine.key1 = i;
                }
                // row i of M: L_i at columns k..k+s-1
                for (int u = 0; u < s; ++u) {
                    M[at(i, k + u) * E] = Li[u][0];
                    if (CPLX) M[at(i, k + u) * E + 1] = Li[u][1];
                }
            } else {
                A[at(i, j) * E] = tr;
                if (CPLX) A[at(i, j) * E + 1] = ti;
                const double v = CPLX ? hypot(tr, ti) : fabs(tr);
                const long long key = (long long)j * n + i;  // the upper-triangle copy (j, i)
                if (fe_better(v, key, mine.mu0, mine.key0)) {
                    mine.mu0 = v;
                    mine.key0 = key;
                }
            }
        }
        // the pivot rows of M: the identity block
        if (gtid < s * s) {
            const int a = (int)(gtid % s), b = (int)(gtid / s);
            M[at(k + a, k + b) * E] = a == b ? 1.0 : 0.0;
            if (CPLX) M[at(k + a, k + b) * E + 1] = 0.0;
        }
        if (gtid == 0) psize[k] = (int8_t)s;
        if (s == 2 && gtid == 1) psize[k + 1] = 0;
        par ^= 1;
        block_max(mine, par);
        k = k1;
        if (!fe_grid_sync(st, nb, wait_ns)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->rank = k;
        st->mu0_init = mu0_init;
    }
}

// G columns from M and the pivot blocks (kept in A's diagonal blocks), rows
// returned to H's order: one thread per (row, pivot column).
template <bool CPLX>
__global__ void fe_finish_kernel(const double *__restrict__ A, const double *__restrict__ M,
                                 int n, int r, const int32_t *__restrict__ perm,
                                 const int8_t *__restrict__ psize, double *__restrict__ G,
                                 int64_t ldg, int8_t *__restrict__ Jout) {
    constexpr int E = CPLX ? 2 : 1;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * r) return;
    const int i = (int)(t % n), c = (int)(t / n);
    const int s = psize[c];
    if (s == 0) return;  // second column of a 2x2 block: written with the first
    auto at = [&](int a, int b) -> int64_t { return (int64_t)b * n + a; };
    const int64_t gi = perm[i];
    if (s == 1) {
        const double d = A[at(c, c) * E];
        const double sc = sqrt(fabs(d));
#pragma unroll
        for (int e = 0; e < E; ++e) G[((int64_t)c * ldg + gi) * E + e] = M[at(i, c) * E + e] * sc;
        if (i == 0) Jout[c] = d > 0.0 ? 1 : -1;
        return;
    }
    // E = [[a, conj(b)], [b, d]] = Q diag(delta) Q^*, delta ascending; columns
    // M_b Q |delta|^(1/2)
    const double a = A[at(c, c) * E], d = A[at(c + 1, c + 1) * E];
    const double br = A[at(c + 1, c) * E], bi = CPLX ? A[at(c + 1, c) * E + 1] : 0.0;
    const double babs = hypot(br, bi);
    const double mid = 0.5 * (a + d), half = 0.5 * (a - d);
    const double rad = hypot(half, babs);
    const double dl = mid - rad, dh = mid + rad;  // delta_1 <= delta_2
    // eigenvector of dh: (cos, e^{i phi} sin) with tan(2 theta) = 2|b| / (a - d)
    const double th = 0.5 * atan2(babs, half);
    const double cs = cos(th), sn = sin(th);
    const double pr = babs > 0.0 ? br / babs : 1.0, pi = babs > 0.0 ? bi / babs : 0.0;
    // q2 = (cs, e^{i phi} sn) for dh; q1 = (-sn, e^{i phi} cs) for dl
    const double m0r = M[at(i, c) * E], m0i = CPLX ? M[at(i, c) * E + 1] : 0.0;
    const double m1r = M[at(i, c + 1) * E], m1i = CPLX ? M[at(i, c + 1) * E + 1] : 0.0;
    // m1 * e^{i phi}
    const double er = m1r * pr - m1i * pi, ei = m1r * pi + m1i * pr;
    const double g1r = -sn * m0r + cs * er, g1i = -sn * m0i + cs * ei;  // M_b q1
    const double g2r = cs * m0r + sn * er, g2i = cs * m0i + sn * ei;    // M_b q2
    const double s1 = sqrt(fabs(dl)), s2 = sqrt(fabs(dh));
    G[((int64_t)c * ldg + gi) * E] = g1r * s1;
    G[((int64_t)(c + 1) * ldg + gi) * E] = g2r * s2;
    if (CPLX) {
        G[((int64_t)c * ldg + gi) * E + 1] = g1i * s1;
        G[((int64_t)(c + 1) * ldg + gi) * E + 1] = g2i * s2;
    }
    if (i == 0) {
        Jout[c] = dl > 0.0 ? 1 : -1;
        Jout[c + 1] = dh > 0.0 ? 1 : -1;
    }
}

template <bool CPLX>
__global__ void fe_copy_kernel(const double *__restrict__ H, int64_t ldh, int n, double *__restrict__ A,
                               int32_t *__restrict__ perm) {
    constexpr int E = CPLX ? 2 : 1;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    const int i = (int)(t % n), j = (int)(t / n);
    if (j == 0) perm[i] = i;
    if (i < j) return;  // only the lower triangle is stored
    A[t * E] = H[((int64_t)j * ldh + i) * E];
    if (CPLX) A[t * E + 1] = i == j ? 0.0 : H[((int64_t)j * ldh + i) * E + 1];
}

}  // namespace

int frontend_factor(bool cplx, const double *H, int64_t ldh, int n, double rank_tol, double *G,
                    int64_t ldg, int8_t *J_host, int32_t *perm_host, int8_t *psize_host,
                    int64_t *rank_host, uint64_t wait_ns, cudaStream_t st) {
    const int E = cplx ? 2 : 1;
    int dev = 0, sms = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return JJ_CUDA_ERROR;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
        return JJ_CUDA_ERROR;
    auto kern = cplx ? fe_eliminate_kernel<true> : fe_eliminate_kernel<false>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FE_THREADS, 0) != cudaSuccess ||
        per_sm < 1)
        return JJ_CUDA_ERROR;
    const int nb = sms * (per_sm < 2 ? per_sm : 2);
    double *A = nullptr, *M = nullptr;
    int32_t *perm = nullptr;
    int8_t *psize = nullptr, *Jd = nullptr;
    FeState *state = nullptr;
    FeMax *bmax = nullptr;
    const size_t nn = (size_t)n * n;
    cudaError_t e = cudaMallocAsync((void **)&A, nn * E * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&M, nn * E * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&perm, (size_t)n * sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&psize, (size_t)n, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&Jd, (size_t)n, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&state, sizeof(FeState), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&bmax, 2 * (size_t)nb * sizeof(FeMax), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(state, 0, sizeof(FeState), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(M, 0, nn * E * sizeof(double), st);
    if (e == cudaSuccess) {
        const unsigned g = (unsigned)((nn + 255) / 256);
        if (cplx)
            fe_copy_kernel<true><<<g, 256, 0, st>>>(H, ldh, n, A, perm);
        else
            fe_copy_kernel<false><<<g, 256, 0, st>>>(H, ldh, n, A, perm);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        void *args[] = {&A, &M, &n, &perm, &psize, &state, &bmax, &rank_tol, &wait_ns};
        e = cudaLaunchCooperativeKernel((const void *)kern, dim3(nb), dim3(FE_THREADS), args, 0, st);
    }
    FeState hs{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, state, sizeof(FeState), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int rc = e == cudaSuccess ? JJ_OK : JJ_CUDA_ERROR;
    if (rc == JJ_OK && hs.err) rc = JJ_DEVICE_TIMEOUT;
    const int r = rc == JJ_OK ? hs.rank : 0;
    if (rc == JJ_OK && r > 0) {
        const unsigned g = (unsigned)(((size_t)n * r + 255) / 256);
        if (cplx)
            fe_finish_kernel<true><<<g, 256, 0, st>>>(A, M, n, r, perm, psize, G, ldg, Jd);
        else
            fe_finish_kernel<false><<<g, 256, 0, st>>>(A, M, n, r, perm, psize, G, ldg, Jd);
        if (cudaGetLastError() != cudaSuccess) rc = JJ_CUDA_ERROR;
    }
    if (rc == JJ_OK) {
        std::vector<int8_t> ps(n);
        if (cudaMemcpyAsync(J_host, Jd, (size_t)r, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(ps.data(), psize, (size_t)n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            (perm_host && cudaMemcpyAsync(perm_host, perm, (size_t)n * sizeof(int32_t),
                                          cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = JJ_CUDA_ERROR;
        if (psize_host)
            for (int c = 0; c < n; ++c) psize_host[c] = c < r ? ps[c] : 0;
    }
    if (rank_host) *rank_host = r;
    cudaFreeAsync(A, st);
    cudaFreeAsync(M, st);
    cudaFreeAsync(perm, st);
    cudaFreeAsync(psize, st);
    cudaFreeAsync(Jd, st);
    cudaFreeAsync(state, st);
    cudaFreeAsync(bmax, st);
    return rc;
}

}  // namespace jj
