// Block update (2.9) on the FP64 pipe: [G_i G_j] <- [G_i G_j] W_P, in place.
//
// Pair descriptor: int32 {off_i, n_i, off_j, n_j}; the k = n_i + n_j pivot
// columns are G[:, off_i + a] for a < n_i and G[:, off_j + a - n_i] after.
// W_P is kmax x kmax column-major at pair * kmax * kmax elements (complex:
// interleaved).
#include "jj_common.cuh"

namespace jj {
namespace {

__device__ __forceinline__ int64_t pivot_col(const int32_t *pd, int a) {
    return a < pd[1] ? (int64_t)pd[0] + a : (int64_t)pd[2] + (a - pd[1]);
}

// ---------------------------------------------------------------------------
// Update, FP64 (2.9): [G_i G_j] <- [G_i G_j] W_P for the rows of one tile. One
// block per (tile of VR rows, pair) computes every output column of its rows,
// so the tile of X is read completely (into shared memory) before any output
// is written: the update is done in place (Gd may equal Gs). W_P is staged
// through shared memory VKA rows at a time. Thread (rg, cg) owns rows
// rg + 8 i and columns cg + 32 j of a chunk of 32 NJ output columns.
// ---------------------------------------------------------------------------
constexpr int VKA = 16;  // rows of W_P per stage

template <bool CPLX, int NJ>
__global__ void __launch_bounds__(256, 2) update_fp64_kernel(const double *Gs, double *Gd, int64_t ld,
                                                           int64_t m, const int32_t *__restrict__ pairs,
                                                           const double *__restrict__ W, int kmax,
                                                           int VR, StepCtl ctl) {
    constexpr int E = CPLX ? 2 : 1;
    constexpr int KW = 32 * NJ;  // output columns per chunk
    extern __shared__ double usm[];
    double *xs = usm;                              // [a][r][e], k x VR
    double *ws = usm + (size_t)kmax * VR * E;      // [a'][c][e], VKA x KW
    const int q = blockIdx.y;
    const int32_t *pd = pairs + 4 * q;
    const int k = pd[1] + pd[3];
    const int64_t mq = pair_rows(ctl, q, m);
    const int64_t l0 = (int64_t)blockIdx.x * VR;
    if (l0 >= mq) return;
    const int64_t l1 = min(mq, l0 + VR);
    if (pair_passthrough(ctl, q)) {
        if (Gd != Gs) pair_copy_rows(CPLX, Gs, Gd, ld, pd, l0, l1, 0, k, threadIdx.x, 256);
        return;
    }
    const int tid = threadIdx.x;
    // Only the columns the inner solve rotated change: W restricted to the
    // others is the identity (their entries of W are exact zeros and ones),
    // so Y_t = X_t W_tt over the rotated set t, with the same bits.
    __shared__ int tcol[128];
    __shared__ int s_nt;
    int kk = k;
    if (ctl.touched && k <= 128) {
        if (tid == 0) {
            const unsigned long long m0 = ctl.touched[2 * q], m1 = ctl.touched[2 * q + 1];
            int nt = 0;
            for (int c = 0; c < k; ++c)
                if (((c < 64 ? m0 >> c : m1 >> (c - 64)) & 1ull) != 0ull) tcol[nt++] = c;
            s_nt = nt;
        }
        __syncthreads();
        kk = s_nt;
        if (kk == 0) return;
    } else {
        for (int c = tid; c < k && c < 128; c += 256) tcol[c] = c;
        __syncthreads();
    }
    auto cmap = [&](int i) -> int { return i < 128 ? tcol[i] : i; };
    for (int idx = tid; idx < kk * VR; idx += 256) {
        const int a = idx / VR, r = idx % VR;
        const int64_t l = l0 + r;
        const int64_t col = pivot_col(pd, cmap(a));
#pragma unroll
        for (int e = 0; e < E; ++e) xs[((size_t)a * VR + r) * E + e] = l < l1 ? Gs[(col * ld + l) * E + e] : 0.0;
    }
    const double *Wp = W + (size_t)q * kmax * kmax * E;
    const int rg = tid & 7, cg = tid >> 3;
    const int nri = VR / 8;  // rows per thread (<= 4)
    for (int c0 = 0; c0 < kk; c0 += KW) {
        double acc[4][NJ][E];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < NJ; ++j)
#pragma unroll
                for (int e = 0; e < E; ++e) acc[i][j][e] = 0.0;
        for (int a0 = 0; a0 < kk; a0 += VKA) {
            __syncthreads();  // X tile complete / previous W stage consumed
            for (int idx = tid; idx < VKA * KW; idx += 256) {
                const int aa = idx % VKA, c = idx / VKA;
                const int a = a0 + aa, b = c0 + c;
                const bool ok = a < kk && b < kk;
#pragma unroll
                for (int e = 0; e < E; ++e)
                    ws[((size_t)aa * KW + c) * E + e] =
                        ok ? Wp[((size_t)cmap(b) * kmax + cmap(a)) * E + e] : 0.0;
            }
            __syncthreads();
            const int na = min(VKA, kk - a0);
            for (int aa = 0; aa < na; ++aa) {
                const double *xa = xs + (size_t)(a0 + aa) * VR * E;
                const double *wa = ws + (size_t)aa * KW * E;
                double w[NJ][E];
#pragma unroll
                for (int j = 0; j < NJ; ++j)
#pragma unroll
                    for (int e = 0; e < E; ++e) w[j][e] = wa[(cg + 32 * j) * E + e];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (i >= nri) break;
                    const int r = rg + 8 * i;
                    if (CPLX) {
                        const double xr = xa[r * 2], xi = xa[r * 2 + 1];
#pragma unroll
                        for (int j = 0; j < NJ; ++j) {
                            acc[i][j][0] = fma(xr, w[j][0], fma(-xi, w[j][E - 1], acc[i][j][0]));
                            acc[i][j][E - 1] = fma(xr, w[j][E - 1], fma(xi, w[j][0], acc[i][j][E - 1]));
                        }
                    } else {
                        const double x = xa[r];
#pragma unroll
                        for (int j = 0; j < NJ; ++j) acc[i][j][0] = fma(x, w[j][0], acc[i][j][0]);
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i >= nri) break;
            const int64_t l = l0 + rg + 8 * i;
            if (l >= l1) continue;
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const int b = c0 + cg + 32 * j;
                if (b < kk) {
                    const int64_t col = pivot_col(pd, cmap(b));
#pragma unroll
                    for (int e = 0; e < E; ++e) Gd[(col * ld + l) * E + e] = acc[i][j][e];
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_update(bool cplx, int gemm, const double *Gs, double *Gd, int64_t ld,
                          int64_t m, const int32_t *pairs, int npairs, const double *W,
                          int kmax, cudaStream_t st, StepCtl ctl) {
    (void)gemm;
    if (npairs <= 0) return cudaSuccess;
    const int E = cplx ? 2 : 1;
    const int nj = kmax <= 32 ? 1 : kmax <= 64 ? 2 : (cplx || kmax <= 128) ? 4 : 8;
    // rows per tile: 32, fewer when the X tile would not fit shared memory
    int vr = 32;
    auto smem = [&](int r) { return sizeof(double) * E * ((size_t)kmax * r + (size_t)VKA * 32 * nj); };
    while (vr > 8 && smem(vr) > 200 * 1024) vr /= 2;
    if (smem(vr) > 227 * 1024) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((m + vr - 1) / vr), npairs);
    const size_t sb = smem(vr);
#define JJ_UPD(C, N)                                                                          \
    do {                                                                                      \
        auto kern = update_fp64_kernel<C, N>;                                                 \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)sb);                                        \
        if (e != cudaSuccess) return e;                                                       \
        kern<<<grid, 256, sb, st>>>(Gs, Gd, ld, m, pairs, W, kmax, vr, ctl);                  \
        return cudaGetLastError();                                                            \
    } while (0)
    if (cplx) {
        if (nj == 1) JJ_UPD(true, 1);
        if (nj == 2) JJ_UPD(true, 2);
        JJ_UPD(true, 4);
    } else {
        if (nj == 1) JJ_UPD(false, 1);
        if (nj == 2) JJ_UPD(false, 2);
        if (nj == 4) JJ_UPD(false, 4);
        JJ_UPD(false, 8);
    }
#undef JJ_UPD
}

}  // namespace jj
