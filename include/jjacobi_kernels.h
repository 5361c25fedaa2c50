/*
 * jjacobi_kernels.h -- building-block entry points of the J-Jacobi library.
 *
 * Each call launches one kernel family of the hot path on device memory, on
 * the given stream (NULL: legacy default stream), asynchronously; the return
 * value reports argument errors and launch errors only (jj_status codes of
 * jjacobi.h). They exist so that each step of the path can be checked on its
 * own against the CPU oracle, and so that callers can assemble custom drivers.
 *
 * Common layouts:
 *   G       column-major m x n, leading dimension ld (elements); complex
 *           values interleaved (re, im).
 *   pairs   int32 [npairs][4] = {off_i, n_i, off_j, n_j}: pivot pair of block
 *           columns G_i = G[:, off_i : off_i+n_i], G_j = G[:, off_j : off_j+n_j]
 *           (Sec. 3.2, (3.5)); k = n_i + n_j <= kmax.
 *   blocks  per pair a column-major kmax x kmax block (ld = kmax) at offset
 *           pair * kmax * kmax elements (A_P, R, W_P).
 *   J       device int8 [n], +-1 (signs of the columns of G).
 *   counters device uint64 [8]: [0] rotations applied (atomic add),
 *           [1] bit pattern of the largest scaled |a_rs| seen (atomic max),
 *           [2] error flags (1: not positive definite, 2: non-finite,
 *           4: device wait expired), [3] pivot pairs evaluated by jjk_inner,
 *           [4] pivot pairs that applied a rotation, [5..7] reserved.
 */
#ifndef JJACOBI_KERNELS_H
#define JJACOBI_KERNELS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* d[c] = ||g_c||^2 for every column c < n (start of a sweep, Alg. 3.2). */
int jjk_column_norms(int32_t dtype, const void *G, int64_t ld, int64_t m, int64_t n,
                     double *d, void *stream);

/* One parallel step of the plain method (K-a): for every pair (r, s) of
 * `pairs` (int32 [npairs][2], column indices; entries >= n are skipped),
 * a_rs = g_r^* g_s; if |a_rs| > tol sqrt(d_r d_s) the rotation of Alg. 3.1
 * (hyp = J_r J_s) updates g_r, g_s (2.13) and the tracked d_r, d_s.
 * Pairs of one call must be disjoint. */
int jjk_plain_step(int32_t dtype, void *G, int64_t ld, int64_t m, int64_t n,
                   const int32_t *pairs, int32_t npairs, const int8_t *J, double *d,
                   double tol, unsigned long long *counters, void *stream);

/* Gram of every pivot pair (K-b, (3.6)): A_p = [G_i G_j]^* [G_i G_j], written as
 * the full Hermitian k x k block (both triangles). gemm (jj_gemm) selects the
 * Gram's form as the solver does: FP64 for JJ_GEMM_FP64; digit products for
 * JJ_GEMM_OZAKI_FP16 and JJ_GEMM_OZAKI_GRAM (JJ_INVALID_ARG when the pivot
 * width exceeds what they take: real width 2 kmax (complex) or kmax (real)
 * above 256; a pivot wider than 64 real columns runs as tiles of 64);
 * JJ_GEMM_AUTO: digit products where they apply, else FP64. Other values:
 * JJ_INVALID_ARG. */
int jjk_gram(int32_t dtype, int32_t gemm, const void *G, int64_t ld, int64_t m,
             const int32_t *pairs, int32_t npairs, double *A, int32_t kmax, void *stream);

/* Inner solve of every pivot pair (K-d): Cholesky A_p = R^* R (R upper; the
 * lower triangle of the block is ignored on input), then the one-sided
 * J-Jacobi method on the columns of R with J_P = diag(J_i, J_j) (Alg. 3.2,
 * inner_block_width 0) or the blocked full-block method (Alg. 3.3, inner
 * blocks of inner_block_width columns), with W_p accumulated from I (3.12).
 * On return A holds R~ = R W_p and W holds W_p. Rotations, the largest scaled
 * off-diagonal and failures go to counters. */
int jjk_inner(int32_t dtype, double *A, double *W, int32_t kmax, const int32_t *pairs,
              int32_t npairs, const int8_t *J, double tol, int32_t inner_max_sweeps,
              int32_t inner_block_width, unsigned long long *counters, void *stream);

/* Block update (K-c, (2.9)): [Gd_i Gd_j] = [Gs_i Gs_j] W_p for every pair
 * (both use ld and the pair's column offsets). Gd may equal Gs (in place: each
 * block reads every row it writes before writing it); otherwise the two must
 * not overlap. gemm: digit products for JJ_GEMM_OZAKI_FP16 (the all-digit
 * form), FP64 for JJ_GEMM_FP64, JJ_GEMM_OZAKI_GRAM and JJ_GEMM_AUTO (as in the
 * solver); other values: JJ_INVALID_ARG. */
int jjk_update(int32_t dtype, int32_t gemm, const void *Gs, void *Gd, int64_t ld,
               int64_t m, const int32_t *pairs, int32_t npairs, const double *W,
               int32_t kmax, void *stream);

/* Eigenpairs (K-f): lambda[c] = J[c] ||g_c||^2, and if U is not NULL
 * u_c = g_c / ||g_c|| (m x n, ldu). */
int jjk_extract(int32_t dtype, const void *G, int64_t ld, int64_t m, int64_t n,
                const int8_t *J, double *lambda, void *U, int64_t ldu, void *stream);

/* The Gram of jjk_gram with gemm = JJ_GEMM_OZAKI_FP16, for callers that cannot
 * allocate device memory (the paper has no counterpart: this is a property of
 * the library, not of the method). Such callers include code running inside a
 * host callback or a driver hook where allocation calls are not allowed, and
 * real-time loops that must not enter an allocator after start-up. jjk_gram
 * takes its scratch from the stream-ordered allocator; this call takes it from
 * one fixed array of device memory inside the library instead (about 8.3 MiB,
 * held by every GPU that loads the library until the process exits).
 *   Limits: npairs * (2 kmax)^2 * 16 bytes (complex) or npairs * kmax^2 * 16
 *   bytes (real) must not exceed 8 MiB, real pivot width (2 kmax complex,
 *   kmax real) <= 64, and ncols <= 65536; larger sizes return JJ_INVALID_ARG.
 *   ncols: number of columns of G; every column a pair names must be < ncols.
 *   The first call on a device looks up the array's device address (with that
 *   device current) and should come before any stream capture.
 *   Every call shares the one array and clears the part it uses before use;
 *   two calls whose work overlaps on the GPU (different streams, or different
 *   host threads without ordering) race on it. No cudaMalloc, cudaFree or
 *   other allocating routine is called. */
int jjk_gram_noalloc(int32_t dtype, const void *G, int64_t ld, int64_t m, const int32_t *pairs,
                     int32_t npairs, double *A, int32_t kmax, int64_t ncols, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* JJACOBI_KERNELS_H */
