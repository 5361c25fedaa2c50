// Blocked form, FP64 kernels: the pivot Gram (3.6) and the inner solve on the
// Cholesky factor (Cholesky (3.8) + one-sided J-Jacobi (3.12) with explicit
// accumulation of W_P). The FP64 block update (2.9) is in jj_update.cu.
//
// Pair descriptor: int32 {off_i, n_i, off_j, n_j}; the k = n_i + n_j pivot
// columns are G[:, off_i + a] for a < n_i and G[:, off_j + a - n_i] after.
// Per-pair blocks (A_P, R, W_P) are kmax x kmax column-major at
// pair * kmax * kmax elements (complex: interleaved).
#include "jj_common.cuh"
#include "jj_digits.cuh"

namespace jj {
namespace {

__device__ __forceinline__ int64_t pivot_col(const int32_t *pd, int a) {
    return a < pd[1] ? (int64_t)pd[0] + a : (int64_t)pd[2] + (a - pd[1]);
}

// ---------------------------------------------------------------------------
// Gram, FP64 on the FP64 pipe: one block per (32 x 32 tile of A_P, pair);
// only tiles on or above the diagonal are formed, the lower triangle is
// written as the conjugate transpose.
// ---------------------------------------------------------------------------
constexpr int GT = 32;   // output tile edge
constexpr int GKR = 16;  // rows of G staged per k-step

template <bool CPLX>
__global__ void __launch_bounds__(256) gram_fp64_kernel(const double *__restrict__ G, int64_t ld,
                                                         int64_t m, const int32_t *__restrict__ pairs,
                                                         double *__restrict__ A, int kmax, StepCtl ctl) {
    constexpr int E = CPLX ? 2 : 1;
    __shared__ double xa[GKR][GT][E];
    __shared__ double xb[GKR][GT][E];
    const int32_t *pd = pairs + 4 * blockIdx.y;
    if (ctl.mod_step) {
        const bool skip = pair_skip_decide(ctl, pd, blockIdx.y);
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl.flags[blockIdx.y] = skip ? kPairSkipped : 0;
        if (skip) return;
    }
    const int k = pd[1] + pd[3];
    // map linear tile index to (ta, tb) with ta <= tb
    int t = blockIdx.x, ta = 0;
    const int T = (kmax + GT - 1) / GT;
    while (t >= T - ta) {
        t -= T - ta;
        ++ta;
    }
    const int tb = ta + t;
    const int a0 = ta * GT, b0 = tb * GT;
    if (a0 >= k || b0 >= k) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2 x 2 outputs each
    double acc[2][2][E];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int e = 0; e < E; ++e) acc[i][j][e] = 0.0;
    // loader: 256 threads load GKR x GT entries of each operand
    const int lr = threadIdx.x / GT * 2;  // 0,2,..,14 (rows, two per thread)
    const int lc = threadIdx.x % GT;
    const int64_t ca = a0 + lc < k ? pivot_col(pd, a0 + lc) : -1;
    const int64_t cb = b0 + lc < k ? pivot_col(pd, b0 + lc) : -1;
    for (int64_t l0 = 0; l0 < m; l0 += GKR) {
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int64_t l = l0 + lr + rr;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                xa[lr + rr][lc][e] = (ca >= 0 && l < m) ? G[(ca * ld + l) * E + e] : 0.0;
                xb[lr + rr][lc][e] = (cb >= 0 && l < m) ? G[(cb * ld + l) * E + e] : 0.0;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int q = 0; q < GKR; ++q) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int a = ty + 16 * i;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int b = tx + 16 * j;
                    if (CPLX) {
                        const double ar = xa[q][a][0], ai = xa[q][a][1];
                        const double br = xb[q][b][0], bi = xb[q][b][1];
                        acc[i][j][0] = fma(ar, br, fma(ai, bi, acc[i][j][0]));
                        acc[i][j][E - 1] = fma(ar, bi, fma(-ai, br, acc[i][j][E - 1]));
                    } else {
                        acc[i][j][0] = fma(xa[q][a][0], xb[q][b][0], acc[i][j][0]);
                    }
                }
            }
        }
        __syncthreads();
    }
    double *Ap = A + (int64_t)blockIdx.y * kmax * kmax * E;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int a = a0 + ty + 16 * i;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int b = b0 + tx + 16 * j;
            // one writer per entry: on a diagonal tile only a <= b (the (b, a)
            // sum is rounded in another order and must not race with it)
            if (a < k && b < k && (ta != tb || a <= b)) {
                Ap[((int64_t)b * kmax + a) * E] = acc[i][j][0];
                if (CPLX) Ap[((int64_t)b * kmax + a) * E + 1] = a == b ? 0.0 : acc[i][j][E - 1];
                if (a != b) {
                    Ap[((int64_t)a * kmax + b) * E] = acc[i][j][0];
                    if (CPLX) Ap[((int64_t)a * kmax + b) * E + 1] = -acc[i][j][E - 1];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Inner solve, one block per pair: Cholesky of A_P into R (upper), then the
// one-sided J-Jacobi method on the k columns of R in the standard round-robin
// parallel order (k/2 disjoint column pairs per inner step, one warp per
// pair), W_P accumulated from I. The tracked diagonal is recomputed at the
// start of each inner sweep (Alg. 3.2). R and W stay in global memory (they are
// L2-resident) and are accessed with .cg loads/stores.
// ---------------------------------------------------------------------------
constexpr int IT = 256;  // threads

template <bool CPLX>
__device__ __forceinline__ void inner_rr_pair(int npl, int step, int q, int &a, int &b) {
    // Standard round-robin (circle) schedule over npl (even) players: player
    // npl-1 is fixed, the others rotate by one each step.
    const int P = npl - 1;
    if (q == 0) {
        a = P;
        b = step;
    } else {
        a = (step + q) % P;
        b = (step - q + P) % P;
    }
}

template <bool CPLX>
__global__ void __launch_bounds__(IT) inner_kernel(double *__restrict__ A, double *__restrict__ Wb,
                                                    int kmax, const int32_t *__restrict__ pairs,
                                                    const int8_t *__restrict__ J, double tol,
                                                    int max_sweeps,
                                                    unsigned long long *__restrict__ counters,
                                                    StepCtl ctl) {
    constexpr int E = CPLX ? 2 : 1;
    if (ctl.flags && (ctl.flags[blockIdx.x] & kPairSkipped)) return;
    extern __shared__ double smem[];
    double *dsh = smem;                        // kmax tracked diagonal
    int *jsh = reinterpret_cast<int *>(dsh + kmax);  // kmax signs
    __shared__ int s_rot, s_fail;
    const int32_t *pd = pairs + 4 * blockIdx.x;
    const int k = pd[1] + pd[3];
    double *R = A + (int64_t)blockIdx.x * kmax * kmax * E;
    double *W = Wb + (int64_t)blockIdx.x * kmax * kmax * E;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int a = tid; a < k; a += IT) jsh[a] = J[pivot_col(pd, a)];
    if (tid == 0) s_fail = 0;
    __syncthreads();
    // --- Cholesky, right-looking, upper: A = R^* R --------------------------
    for (int j = 0; j < k; ++j) {
        __shared__ double piv;
        if (tid == 0) {
            const double ajj = R[((int64_t)j * kmax + j) * E];
            if (!(ajj > 0.0) || !isfinite(ajj)) {
                s_fail = 1;
                piv = 1.0;
            } else {
                piv = sqrt(ajj);
            }
        }
        __syncthreads();
        if (s_fail) break;
        const double rjj = piv, inv = 1.0 / rjj;
        // row j of R: r_jl = a_jl / r_jj for l > j
        for (int l = j + 1 + tid; l < k; l += IT) {
#pragma unroll
            for (int e = 0; e < E; ++e) R[((int64_t)l * kmax + j) * E + e] *= inv;
        }
        if (tid == 0) {
            R[((int64_t)j * kmax + j) * E] = rjj;
            if (CPLX) R[((int64_t)j * kmax + j) * E + 1] = 0.0;
        }
        __syncthreads();
        // trailing update of the upper triangle: a_{l1 l2} -= conj(r_{j l1}) r_{j l2}
        const int rem = k - j - 1;
        const int total = rem * (rem + 1) / 2;
        for (int t = tid; t < total; t += IT) {
            // t -> (l1 <= l2) over the remaining upper triangle, column-wise
            int l2 = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
            while ((l2 + 1) * (l2 + 2) / 2 <= t) ++l2;
            while (l2 * (l2 + 1) / 2 > t) --l2;
            const int l1 = t - l2 * (l2 + 1) / 2;
            const int c1 = j + 1 + l1, c2 = j + 1 + l2;
            if (CPLX) {
                const double ur = R[((int64_t)c1 * kmax + j) * E], ui = R[((int64_t)c1 * kmax + j) * E + 1];
                const double vr = R[((int64_t)c2 * kmax + j) * E], vi = R[((int64_t)c2 * kmax + j) * E + 1];
                double *dst = R + ((int64_t)c2 * kmax + c1) * E;
                dst[0] -= ur * vr + ui * vi;
                dst[1] -= ur * vi - ui * vr;
            } else {
                R[(int64_t)c2 * kmax + c1] -= R[(int64_t)c1 * kmax + j] * R[(int64_t)c2 * kmax + j];
            }
        }
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) {
            atomicOr(&counters[kCntErr], kErrNotPosdef);
            pair_record(ctl, pd, blockIdx.x, false, true);
            pair_flag_prob(ctl, blockIdx.x, kErrNotPosdef);
        }
        // leave W = I so that the update is the identity
        for (int64_t t = tid; t < (int64_t)k * k; t += IT) {
            const int a = (int)(t % k), b = (int)(t / k);
            W[((int64_t)b * kmax + a) * E] = a == b ? 1.0 : 0.0;
            if (CPLX) W[((int64_t)b * kmax + a) * E + 1] = 0.0;
        }
        return;
    }
    // zero the strictly lower triangle of R, W = I
    for (int64_t t = tid; t < (int64_t)k * k; t += IT) {
        const int a = (int)(t % k), b = (int)(t / k);
        if (a > b) {
            R[((int64_t)b * kmax + a) * E] = 0.0;
            if (CPLX) R[((int64_t)b * kmax + a) * E + 1] = 0.0;
        }
        W[((int64_t)b * kmax + a) * E] = a == b ? 1.0 : 0.0;
        if (CPLX) W[((int64_t)b * kmax + a) * E + 1] = 0.0;
    }
    __syncthreads();
    // --- inner one-sided J-Jacobi on the columns of R ------------------------
    const int npl = k + (k & 1);
    unsigned long long total_rot = 0;
    double maxoff = 0.0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        // d_c = ||r_c||^2
        for (int c = warp; c < k; c += IT / 32) {
            double acc = 0.0;
            for (int l = lane; l < k; l += 32) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const double v = R[((int64_t)c * kmax + l) * E + e];
                    acc = fma(v, v, acc);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) dsh[c] = acc;
        }
        if (tid == 0) s_rot = 0;
        __syncthreads();
        maxoff = 0.0;
        for (int step = 0; step < npl - 1; ++step) {
            for (int q = warp; q < npl / 2; q += IT / 32) {
                int a, b;
                inner_rr_pair<CPLX>(npl, step, q, a, b);
                if (a >= k || b >= k) continue;
                if (a > b) {
                    const int t = a;
                    a = b;
                    b = t;
                }
                double sr = 0.0, si = 0.0;
                double *ra = R + (int64_t)a * kmax * E, *rb = R + (int64_t)b * kmax * E;
                for (int l = lane; l < k; l += 32) {
                    if (CPLX) {
                        const double xr = ra[2 * l], xi = ra[2 * l + 1];
                        const double yr = rb[2 * l], yi = rb[2 * l + 1];
                        sr = fma(xr, yr, fma(xi, yi, sr));
                        si = fma(xr, yi, fma(-xi, yr, si));
                    } else {
                        sr = fma(ra[l], rb[l], sr);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sr += __shfl_xor_sync(0xffffffffu, sr, o);
                    si += __shfl_xor_sync(0xffffffffu, si, o);
                }
                const double da = dsh[a], db = dsh[b];
                const double absa = CPLX ? sqrt(sr * sr + si * si) : fabs(sr);
                const double rel = absa / sqrt(da * db);
                if (!isfinite(rel)) {
                    if (lane == 0) {
                        atomicOr(&counters[kCntErr], kErrNonfinite);
                        pair_flag_prob(ctl, blockIdx.x, kErrNonfinite);
                    }
                    continue;
                }
                maxoff = fmax(maxoff, rel);
                if (!(rel > tol)) continue;
                Rot Q;
                const bool ok = rotation(da, db, sr, si, jsh[a] * jsh[b], CPLX, Q);
                if (!ok) {
                    if (lane == 0) {
                        atomicOr(&counters[kCntErr], kErrNotPosdef);
                        pair_flag_prob(ctl, blockIdx.x, kErrNotPosdef);
                    }
                    continue;
                }
                if (lane == 0) {
                    dsh[a] = Q.dr;
                    dsh[b] = Q.ds;
                    atomicAdd(&s_rot, 1);
                }
                double *wa = W + (int64_t)a * kmax * E, *wb = W + (int64_t)b * kmax * E;
                for (int l = lane; l < k; l += 32) {
                    if (CPLX) {
                        rot_apply_c(Q, ra[2 * l], ra[2 * l + 1], rb[2 * l], rb[2 * l + 1]);
                        rot_apply_c(Q, wa[2 * l], wa[2 * l + 1], wb[2 * l], wb[2 * l + 1]);
                    } else {
                        rot_apply_r(Q, ra[l], rb[l]);
                        rot_apply_r(Q, wa[l], wb[l]);
                    }
                }
            }
            __syncthreads();
        }
        const int rot = s_rot;
        total_rot += (unsigned long long)rot;
        __syncthreads();
        if (rot == 0) break;
    }
    // block max of maxoff
    __shared__ double smax[IT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxoff = fmax(maxoff, __shfl_xor_sync(0xffffffffu, maxoff, o));
    if (lane == 0) smax[warp] = maxoff;
    __syncthreads();
    if (tid == 0) {
        double mo = 0.0;
        for (int w = 0; w < IT / 32; ++w) mo = fmax(mo, smax[w]);
        atomic_max_nonneg(&counters[kCntMaxOff], mo);
        if (total_rot) atomicAdd(&counters[kCntRot], total_rot);
        atomicAdd(&counters[kCntPairs], 1ull);
        if (total_rot) atomicAdd(&counters[kCntPairsRot], 1ull);
        pair_record(ctl, pd, blockIdx.x, total_rot > 0, false);
        pair_count_prob(ctl, blockIdx.x, total_rot);
    }
}

// ---------------------------------------------------------------------------
// Inner solve with R and W resident in shared memory (pivot order k <= KMAX).
// Cholesky (right-looking, upper) in place, then one-sided J-Jacobi sweeps in
// the standard round-robin parallel order: each warp owns one column pair of
// an inner step (lane l holds rows l, l+32, ...), forms the dot product with
// shuffles, lane 0 computes the rotation (Alg. 3.1) and the warp rotates the R
// and W columns. A block barrier separates inner steps.
// ---------------------------------------------------------------------------
constexpr int ST = 512;  // threads per block
constexpr int SW = ST / 32;

template <bool CPLX, int ROWS, bool OFFD>
__global__ void __launch_bounds__(ST) inner_smem_kernel(
    double *__restrict__ A, double *__restrict__ Wb, int kmax, const int32_t *__restrict__ pairs,
    const int8_t *__restrict__ J, double tol, int max_sweeps,
    unsigned long long *__restrict__ counters, StepCtl ctl, UpdDigits ud, int pass, int special) {
    constexpr int E = CPLX ? 2 : 1;
    extern __shared__ double2 smem4[];
    double *sm = reinterpret_cast<double *>(smem4);
    const int32_t *pd = pairs + 4 * blockIdx.x;
    if (ctl.flags && (ctl.flags[blockIdx.x] & kPairSkipped)) return;
    const int k = pd[1] + pd[3];
    const int ldr = k;  // smem leading dimension (entries)
    double *R = sm;                              // k x k entries
    double *W = R + (size_t)k * ldr * E;         // k x k entries
    double *dsh = W + (size_t)k * ldr * E;       // k
    double *qsh = dsh + kmax;                    // per-step dots and rotation parameters
    int *jsh = reinterpret_cast<int *>(qsh + 2 * 64 + 2 * 7 * 64);
    __shared__ int s_rot, s_fail;
    __shared__ double s_piv;
    __shared__ double s_max[SW];
    __shared__ unsigned char s_tcol[128];  // column rotated (one writer per column and step)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double *Ag = A + (int64_t)blockIdx.x * kmax * kmax * E;
    for (int a = tid; a < k; a += ST) jsh[a] = J[pivot_col(pd, a)];
    if (tid < 128) s_tcol[tid] = 0;
    // load the upper triangle of A_P, zero below
    for (int t = tid; t < k * k; t += ST) {
        const int a = t % k, b = t / k;
#pragma unroll
        for (int e = 0; e < E; ++e)
            R[((size_t)b * ldr + a) * E + e] = a <= b ? Ag[((int64_t)b * kmax + a) * E + e] : 0.0;
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    int j0 = 0;  // first column of the right-looking Cholesky below
    if (special && pd[3] > 0) {
        // A pivot of the form (3.7), its diagonal blocks diagonal (their
        // off-diagonal entries, at most tol sqrt(a_rr a_ss), are taken as zero):
        // R_ii = sqrt(Lambda_ii) (3.9), R_ij = R_ii^{-1} A_ij (3.10), and the
        // trailing block gets Lambda_jj - R_ij^* R_ij (3.11), whose Cholesky
        // factor R_jj the loop below computes.
        const int ni = pd[1], nj = pd[3];
        for (int a = tid; a < ni; a += ST) {
            const double ajj = R[((size_t)a * ldr + a) * E];
            const bool ok = ajj > 0.0 && isfinite(ajj);
            dsh[a] = ok ? sqrt(ajj) : 1.0;
            if (!ok) s_fail = 1;
        }
        __syncthreads();
        if (!s_fail) {
            for (int t = tid; t < ni * k; t += ST) {
                const int r = t % ni, cc = t / ni;
                double *dst = R + ((size_t)cc * ldr + r) * E;
                if (cc < ni) {
                    dst[0] = r == cc ? dsh[r] : 0.0;
                    if (CPLX) dst[1] = 0.0;
                } else {
                    const double inv = 1.0 / dsh[r];
#pragma unroll
                    for (int e = 0; e < E; ++e) dst[e] *= inv;
                }
            }
            __syncthreads();
            for (int t = tid; t < nj * nj; t += ST) {
                const int c1 = ni + t % nj, c2 = ni + t / nj;
                if (c1 > c2) continue;
                double sr = c1 == c2 ? R[((size_t)c1 * ldr + c1) * E] : 0.0, si = 0.0;
                for (int r = 0; r < ni; ++r) {
                    if (CPLX) {
                        const double ur = R[((size_t)c1 * ldr + r) * 2], ui = R[((size_t)c1 * ldr + r) * 2 + 1];
                        const double vr = R[((size_t)c2 * ldr + r) * 2], vi = R[((size_t)c2 * ldr + r) * 2 + 1];
                        sr -= fma(ur, vr, ui * vi);
                        si -= fma(ur, vi, -ui * vr);
                    } else {
                        sr -= R[(size_t)c1 * ldr + r] * R[(size_t)c2 * ldr + r];
                    }
                }
                R[((size_t)c2 * ldr + c1) * E] = sr;
                if (CPLX) R[((size_t)c2 * ldr + c1) * E + 1] = si;
            }
        }
        __syncthreads();
        j0 = s_fail ? k : ni;
    }
    // Cholesky A = R^* R (upper), right-looking
    for (int j = j0; j < k; ++j) {
        if (tid == 0) {
            const double ajj = R[((size_t)j * ldr + j) * E];
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
        for (int l = j + 1 + tid; l < k; l += ST) {
#pragma unroll
            for (int e = 0; e < E; ++e) R[((size_t)l * ldr + j) * E + e] *= inv;
        }
        if (tid == 0) {
            R[((size_t)j * ldr + j) * E] = rjj;
            if (CPLX) R[((size_t)j * ldr + j) * E + 1] = 0.0;
        }
        __syncthreads();
        const int rem = k - j - 1;
        // trailing update: column c2 of the remaining block handled by threads
        for (int t = tid; t < rem * rem; t += ST) {
            const int c1 = j + 1 + t % rem, c2 = j + 1 + t / rem;
            if (c1 > c2) continue;
            if (CPLX) {
                const double ur = R[((size_t)c1 * ldr + j) * 2], ui = R[((size_t)c1 * ldr + j) * 2 + 1];
                const double vr = R[((size_t)c2 * ldr + j) * 2], vi = R[((size_t)c2 * ldr + j) * 2 + 1];
                double *dst = R + ((size_t)c2 * ldr + c1) * 2;
                dst[0] -= fma(ur, vr, ui * vi);
                dst[1] -= fma(ur, vi, -ui * vr);
            } else {
                R[(size_t)c2 * ldr + c1] -= R[(size_t)c1 * ldr + j] * R[(size_t)c2 * ldr + j];
            }
        }
        __syncthreads();
    }
    double *Rg = A + (int64_t)blockIdx.x * kmax * kmax * E;
    double *Wg = Wb + (int64_t)blockIdx.x * kmax * kmax * E;
    if (s_fail) {
        if (tid == 0) {
            atomicOr(&counters[kCntErr], kErrNotPosdef);
            pair_record(ctl, pd, blockIdx.x, false, true);
            pair_flag_prob(ctl, blockIdx.x, kErrNotPosdef);
            if (ctl.touched) {
                ctl.touched[2 * blockIdx.x] = 0ull;
                ctl.touched[2 * blockIdx.x + 1] = 0ull;
            }
        }
        for (int t = tid; t < k * k; t += ST) {
            const int a = t % k, b = t / k;
            Wg[((int64_t)b * kmax + a) * E] = a == b ? 1.0 : 0.0;
            if (CPLX) Wg[((int64_t)b * kmax + a) * E + 1] = 0.0;
        }
        return;
    }
    // zero the strictly lower triangle of R (left over from the upper loads), W = I
    for (int t = tid; t < k * k; t += ST) {
        const int a = t % k, b = t / k;
        if (a > b) {
#pragma unroll
            for (int e = 0; e < E; ++e) R[((size_t)b * ldr + a) * E + e] = 0.0;
        }
        W[((size_t)b * ldr + a) * E] = a == b ? 1.0 : 0.0;
        if (CPLX) W[((size_t)b * ldr + a) * E + 1] = 0.0;
    }
    __syncthreads();
    const int npl = k + (k & 1);
    const int P = npl - 1;
    // Passes (Sec. 5.3): pass 0 (full block, 2F) repeats round-robin sweeps
    // over all column pairs of R until one applies no rotation; pass 2 is one
    // such sweep; pass 1 (block-oriented, 2B, after the first step of a sweep)
    // annihilates the off-diagonal block once: round rho pairs column r of the
    // first block with column (r + rho) mod max(n_i, n_j) of the second.
    const int ni = pd[1], nj = pd[3];
    constexpr bool offd = OFFD;  // pass 1 (compile-time: the full passes keep the plain mapping)
    const int NB = ni > nj ? ni : nj;
    const int S = offd ? NB : P;            // inner steps per pass
    const int nq = offd ? ni : npl / 2;     // column pairs per inner step (<= 64)
    const int npass = pass == 0 ? max_sweeps : 1;
    auto pair_at = [&](int st, int qi, int &a, int &b) -> bool {
        if constexpr (offd) {
            const int s2 = (qi + st) % NB;
            a = qi;
            b = ni + s2;
            return qi < ni && s2 < nj;
        }
        a = qi == 0 ? P : (st + qi) % P;
        b = qi == 0 ? st : (st - qi + P) % P;
        if (a > b) { const int t = a; a = b; b = t; }
        return b < k;
    };
    unsigned long long total_rot = 0;
    double maxoff = 0.0;
    // per-step scratch: dot products and rotation parameters of every pair
    double *sdot = qsh;                       // [nq][2]
    double *spar0 = qsh + 2 * 64;             // [2][nq][7]: ce_re ce_im se_re se_im c hs flag
    // Rotations of W are needed only at the end, so the W part of step s is
    // applied by warps 1.. while warp 0 computes the parameters of step s + 1.
    auto apply_w = [&](int st, const double *par, int w0, int nw) {
        for (int qi = w0; qi < nq; qi += nw) {
            const double *pp = par + 7 * qi;
            if (pp[6] == 0.0) continue;
            int a, b;
            pair_at(st, qi, a, b);
            Rot Q;
            Q.ce_re = pp[0]; Q.ce_im = pp[1]; Q.se_re = pp[2]; Q.se_im = pp[3]; Q.c = pp[4]; Q.hs = pp[5];
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                const int l = lane + 32 * i;
                if (l < k) {
                    if (CPLX) {
                        double2 u = *reinterpret_cast<const double2 *>(W + ((size_t)a * ldr + l) * 2);
                        double2 v = *reinterpret_cast<const double2 *>(W + ((size_t)b * ldr + l) * 2);
                        rot_apply_c(Q, u.x, u.y, v.x, v.y);
                        *reinterpret_cast<double2 *>(W + ((size_t)a * ldr + l) * 2) = u;
                        *reinterpret_cast<double2 *>(W + ((size_t)b * ldr + l) * 2) = v;
                    } else {
                        double u = W[(size_t)a * ldr + l], v = W[(size_t)b * ldr + l];
                        rot_apply_r(Q, u, v);
                        W[(size_t)a * ldr + l] = u;
                        W[(size_t)b * ldr + l] = v;
                    }
                }
            }
        }
    };
    for (int sweep = 0; sweep < npass; ++sweep) {
        for (int c = warp; c < k; c += SW) {
            double acc = 0.0;
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                const int l = lane + 32 * i;
                if (l < k) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const double v = R[((size_t)c * ldr + l) * E + e];
                        acc = fma(v, v, acc);
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) dsh[c] = acc;
        }
        if (tid == 0) s_rot = 0;
        __syncthreads();
        int my_rot = 0;
        for (int step = 0; step < S; ++step) {
            // (1) dot products a_ab = r_a^* r_b: one warp per pair, lanes over rows
            for (int qi = warp; qi < nq; qi += SW) {
                int a, b;
                const bool valid = pair_at(step, qi, a, b);
                double sr = 0.0, si = 0.0;
                if (valid) {
#pragma unroll
                    for (int i = 0; i < ROWS; ++i) {
                        const int l = lane + 32 * i;
                        if (l < k) {
                            if (CPLX) {
                                const double2 u = *reinterpret_cast<const double2 *>(R + ((size_t)a * ldr + l) * 2);
                                const double2 v = *reinterpret_cast<const double2 *>(R + ((size_t)b * ldr + l) * 2);
                                sr = fma(u.x, v.x, fma(u.y, v.y, sr));
                                si = fma(u.x, v.y, fma(-u.y, v.x, si));
                            } else {
                                sr = fma(R[(size_t)a * ldr + l], R[(size_t)b * ldr + l], sr);
                            }
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        sr += __shfl_xor_sync(0xffffffffu, sr, o);
                        if (CPLX) si += __shfl_xor_sync(0xffffffffu, si, o);
                    }
                }
                if (lane == 0) {
                    sdot[2 * qi] = sr;
                    sdot[2 * qi + 1] = si;
                }
            }
            __syncthreads();
            // (2) rotation parameters of all pairs of the step at once: warp 0,
            // one lane per pair (the FP64 sequences run once per step, not once
            // per pair); meanwhile the other warps rotate W for the previous step
            double *spar = spar0 + 7 * 64 * (step & 1);
            if (warp != 0 && step > 0) apply_w(step - 1, spar0 + 7 * 64 * ((step - 1) & 1), warp - 1, SW - 1);
            if (warp == 0) {
                for (int qi = lane; qi < nq; qi += 32) {
                    int a, b;
                    const bool valid = pair_at(step, qi, a, b);
                    double flag = 0.0;
                    if (valid) {
                        const double sr = sdot[2 * qi], si = sdot[2 * qi + 1];
                        const double da = dsh[a], db = dsh[b];
                        const double absa = CPLX ? sqrt(sr * sr + si * si) : fabs(sr);
                        const double rel = absa / sqrt(da * db);
                        if (!isfinite(rel)) {
                            atomicOr(&counters[kCntErr], kErrNonfinite);
                            pair_flag_prob(ctl, blockIdx.x, kErrNonfinite);
                        } else {
                            maxoff = fmax(maxoff, rel);
                            if (rel > tol) {
                                Rot Q;
                                if (rotation(da, db, sr, si, jsh[a] * jsh[b], CPLX, Q)) {
                                    double *pp = spar + 7 * qi;
                                    pp[0] = Q.ce_re; pp[1] = Q.ce_im; pp[2] = Q.se_re; pp[3] = Q.se_im;
                                    pp[4] = Q.c; pp[5] = Q.hs;
                                    dsh[a] = Q.dr;
                                    dsh[b] = Q.ds;
                                    flag = 1.0;
                                    ++my_rot;
                                    s_tcol[a] = 1;
                                    s_tcol[b] = 1;
                                } else {
                                    atomicOr(&counters[kCntErr], kErrNotPosdef);
                                    pair_flag_prob(ctl, blockIdx.x, kErrNotPosdef);
                                }
                            }
                        }
                    }
                    spar[7 * qi + 6] = flag;
                }
            }
            __syncthreads();
            // (3) apply to R: one warp per pair, lanes over rows
            for (int qi = warp; qi < nq; qi += SW) {
                const double *pp = spar + 7 * qi;
                if (pp[6] == 0.0) continue;
                int a, b;
                pair_at(step, qi, a, b);
                Rot Q;
                Q.ce_re = pp[0]; Q.ce_im = pp[1]; Q.se_re = pp[2]; Q.se_im = pp[3]; Q.c = pp[4]; Q.hs = pp[5];
#pragma unroll
                for (int i = 0; i < ROWS; ++i) {
                    const int l = lane + 32 * i;
                    if (l < k) {
                        if (CPLX) {
                            double2 u = *reinterpret_cast<const double2 *>(R + ((size_t)a * ldr + l) * 2);
                            double2 v = *reinterpret_cast<const double2 *>(R + ((size_t)b * ldr + l) * 2);
                            rot_apply_c(Q, u.x, u.y, v.x, v.y);
                            *reinterpret_cast<double2 *>(R + ((size_t)a * ldr + l) * 2) = u;
                            *reinterpret_cast<double2 *>(R + ((size_t)b * ldr + l) * 2) = v;
                        } else {
                            double u = R[(size_t)a * ldr + l], v = R[(size_t)b * ldr + l];
                            rot_apply_r(Q, u, v);
                            R[(size_t)a * ldr + l] = u;
                            R[(size_t)b * ldr + l] = v;
                        }
                    }
                }
            }
            __syncthreads();
        }
        // W part of the pass's last step
        apply_w(S - 1, spar0 + 7 * 64 * ((S - 1) & 1), warp, SW);
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) my_rot += __shfl_xor_sync(0xffffffffu, my_rot, o);
            if (lane == 0 && my_rot) atomicAdd(&s_rot, my_rot);
        }
        __syncthreads();
        const int rot = s_rot;
        total_rot += (unsigned long long)rot;
        __syncthreads();
        if (rot == 0) break;
    }
    // Operand of the digit-product update: the digits of D (W2 - I), W2 the real
    // form of W on the update's positions, D the column exponents of the pivot
    // columns (jj_digits.cuh).
    if (ud.img && total_rot > 0) {
        __shared__ int s_xexp[kUdPositions], s_wexp[kUdPositions];
        for (int a = tid; a < kUdPositions; a += ST) {
            const int c = CPLX ? (a & 31) : a;
            s_xexp[a] = c < k ? ud.cexp[pivot_col(pd, c)] : -1021;
        }
        __syncthreads();
        auto wacc = [&](int rr, int cc, int part) -> double { return W[((size_t)cc * ldr + rr) * E + part]; };
        ud_wimage_build<CPLX>(wacc, k, k, true, s_xexp, s_wexp, ud.slices,
                              ud.img + (size_t)blockIdx.x * ud.slices * kUpdSliceBytes,
                              ud.wexp + (size_t)blockIdx.x * kUdPositions, tid, ST);
    }
    // write back R~ and W
    for (int t = tid; t < k * k; t += ST) {
        const int a = t % k, b = t / k;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            Rg[((int64_t)b * kmax + a) * E + e] = R[((size_t)b * ldr + a) * E + e];
            Wg[((int64_t)b * kmax + a) * E + e] = W[((size_t)b * ldr + a) * E + e];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxoff = fmax(maxoff, __shfl_xor_sync(0xffffffffu, maxoff, o));
    if (lane == 0) s_max[warp] = maxoff;
    __syncthreads();
    if (tid == 0) {
        double mo = 0.0;
        for (int w = 0; w < SW; ++w) mo = fmax(mo, s_max[w]);
        atomic_max_nonneg(&counters[kCntMaxOff], mo);
        if (total_rot) atomicAdd(&counters[kCntRot], total_rot);
        atomicAdd(&counters[kCntPairs], 1ull);
        if (total_rot) atomicAdd(&counters[kCntPairsRot], 1ull);
        pair_record(ctl, pd, blockIdx.x, total_rot > 0, false);
        pair_count_prob(ctl, blockIdx.x, total_rot);
        if (ctl.touched) {
            unsigned long long m0 = 0ull, m1 = 0ull;
            for (int c = 0; c < k && c < 128; ++c)
                if (s_tcol[c]) {
                    if (c < 64) m0 |= 1ull << c;
                    else m1 |= 1ull << (c - 64);
                }
            ctl.touched[2 * blockIdx.x] = m0;
            ctl.touched[2 * blockIdx.x + 1] = m1;
        }
    }
}

size_t inner_smem_bytes(bool cplx, int kmax) {
    const int E = cplx ? 2 : 1;
    return sizeof(double) * ((size_t)2 * kmax * kmax * E + kmax + 2 * 64 + 2 * 7 * 64) +
           sizeof(int) * kmax + 64;
}

}  // namespace

cudaError_t launch_gram(bool cplx, int gemm, const double *G, int64_t ld, int64_t m,
                        const int32_t *pairs, int npairs, double *A, int kmax,
                        cudaStream_t st, StepCtl ctl) {
    (void)gemm;
    if (npairs <= 0) return cudaSuccess;
    const int T = (kmax + GT - 1) / GT;
    dim3 grid(T * (T + 1) / 2, npairs);
    if (cplx)
        gram_fp64_kernel<true><<<grid, 256, 0, st>>>(G, ld, m, pairs, A, kmax, ctl);
    else
        gram_fp64_kernel<false><<<grid, 256, 0, st>>>(G, ld, m, pairs, A, kmax, ctl);
    return cudaGetLastError();
}

cudaError_t launch_inner(bool cplx, double *A, double *W, int kmax, const int32_t *pairs,
                         int npairs, const int8_t *J, double tol, int inner_max_sweeps,
                         int inner_block, unsigned long long *counters, cudaStream_t st,
                         StepCtl ctl, UpdDigits ud, int pass, bool special) {
    (void)inner_block;
    if (npairs <= 0) return cudaSuccess;
    // Shared-memory resident form when R and W fit (227 KB per block).
    const size_t smb = inner_smem_bytes(cplx, kmax);
    if (smb <= 227 * 1024 && kmax <= 128) {
#define JJ_INNER_SMEM(C, RW)                                                                  \
    do {                                                                                      \
        auto kern = pass == 1 ? inner_smem_kernel<C, RW, true> : inner_smem_kernel<C, RW, false>; \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)smb);                                       \
        if (e != cudaSuccess) return e;                                                       \
        kern<<<npairs, ST, smb, st>>>(A, W, kmax, pairs, J, tol, inner_max_sweeps, counters, ctl, ud, pass, \
                                      special ? 1 : 0);                                        \
        return cudaGetLastError();                                                            \
    } while (0)
        const int rows = (kmax + 31) / 32;
        if (cplx) {
            if (rows <= 1) JJ_INNER_SMEM(true, 1);
            if (rows <= 2) JJ_INNER_SMEM(true, 2);
            if (rows <= 3) JJ_INNER_SMEM(true, 3);
        } else {
            if (rows <= 1) JJ_INNER_SMEM(false, 1);
            if (rows <= 2) JJ_INNER_SMEM(false, 2);
            if (rows <= 3) JJ_INNER_SMEM(false, 3);
            if (rows <= 4) JJ_INNER_SMEM(false, 4);
        }
#undef JJ_INNER_SMEM
    }
    if (pass != 0 || special) return cudaErrorNotSupported;  // single passes and (3.9)-(3.11) need the shared-memory form
    const size_t sh = (size_t)kmax * sizeof(double) + (size_t)kmax * sizeof(int);
    if (cplx)
        inner_kernel<true><<<npairs, IT, sh, st>>>(A, W, kmax, pairs, J, tol, inner_max_sweeps, counters, ctl);
    else
        inner_kernel<false><<<npairs, IT, sh, st>>>(A, W, kmax, pairs, J, tol, inner_max_sweeps, counters, ctl);
    return cudaGetLastError();
}

bool inner_single_pass_supported(bool cplx, int kmax) {
    return inner_smem_bytes(cplx, kmax) <= 227 * 1024 && kmax <= 128 &&
           (kmax + 31) / 32 <= (cplx ? 3 : 4);
}

}  // namespace jj
