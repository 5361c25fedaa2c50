/*
 * jjacobi.h -- C ABI of the GB300 one-sided hyperbolic (J-)Jacobi eigensolver.
 *
 * Problem (Sec. 2.2, (2.5)-(2.6); Alg. 5.2 "Parallel_Jacobi"): given a full
 * column rank factor G (m x n, m >= n) and J = diag(+-1) with H = G J G^*,
 * compute the eigenpairs of H belonging to its nonzero eigenvalues by the
 * one-sided J-Jacobi method: J-unitary plane rotations from the right on G
 * ((2.9), trigonometric when J_rr = J_ss, hyperbolic otherwise (2.7)) until the
 * columns of G~ = G W are orthogonal to working precision (2.10); then
 *     lambda_i = J_ii ||g~_i||^2,   u_i = g~_i / ||g~_i||    (Alg. 5.2, end).
 *
 * Forms:
 *   block_width == 0  plain, non-blocked method (Algs. 3.1/3.2) with the
 *                     round-robin parallel order over single columns.
 *   block_width  > 0  blocked full-block method (Sec. 3.3, Alg. 5.2 case 2F)
 *                     (block_width == JJ_BLOCK_AUTO: the same, width autotuned):
 *                     per parallel step, for every block pair (i, j):
 *                     Gram A_P = [G_i G_j]^*[G_i G_j] (3.6), Cholesky
 *                     A_P = R^* R (3.8), inner J-Jacobi R W_P = U Sigma with W_P
 *                     accumulated (3.12), update [G_i G_j] <- [G_i G_j] W_P (2.9).
 *   inner_block_width > 0   three-level form (Sec. 5.1, case 3F): the inner
 *                     J-Jacobi on R is itself blocked (Alg. 3.3).
 *
 * Conventions (all entry points):
 *   - Matrices are column-major with a leading dimension (ld >= rows), as in
 *     the paper's Fortran (Sec. 2.3). Complex values are interleaved
 *     (re, im) pairs of doubles (C99 double complex layout).
 *   - "device" pointers are CUDA device (or managed) memory of the current
 *     device; "host" pointers are ordinary host memory (pinned is faster).
 *   - J is a host array of n int8 entries, each +1 or -1.
 *   - Every call returns a status (jj_status); no exception crosses the ABI.
 *     On failure, output buffers may hold partial results.
 *   - A handle is used by one host thread at a time; different handles are
 *     independent. Work is enqueued on the handle's stream; calls that return
 *     results to the host synchronise that stream.
 */
#ifndef JJACOBI_H
#define JJACOBI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define JJACOBI_VERSION 10000 /* 1.0.0 */

typedef struct jj_ctx *jj_handle;

/* Element type of G. */
typedef enum { JJ_F64 = 0, JJ_C128 = 1 } jj_dtype;

/* Parallel block-pivot strategy (Sec. 4): modified round-robin (Alg. 4.3,
 * nbl - 1 steps per sweep) or modified modulus (Alg. 4.2, nbl steps, the
 * blocks on the p-th superdiagonal transformed twice). */
typedef enum { JJ_ORDER_ROUND_ROBIN = 0, JJ_ORDER_MODULUS = 1 } jj_order;

/* How the blocked form computes its two dense contractions (Gram (3.6) and
 * update (2.9)):
 *   JJ_GEMM_FP64        both on the FP64 pipe;
 *   JJ_GEMM_OZAKI_FP16  both as sums of exact fp16 digit products on the
 *                       tensor cores (tcgen05), recombined in integers; the
 *                       update carries one exponent per row and per column,
 *                       and with its default 11 balanced 8-bit digits
 *                       (88 bits) per operand its error stays within FP64's
 *                       per-entry bound on strongly graded inputs;
 *   JJ_GEMM_OZAKI_GRAM  the Gram as digit products, the update in FP64;
 *   JJ_GEMM_AUTO        JJ_GEMM_OZAKI_GRAM when the pivot fits the digit
 *                       kernels, else FP64.
 * The digit kernels take real pivot widths (2 kmax complex, kmax real) up to
 * 256, as 64 x 64 tiles above 64. */
typedef enum {
    JJ_GEMM_FP64 = 0,
    JJ_GEMM_OZAKI_FP16 = 1,
    JJ_GEMM_OZAKI_GRAM = 2,
    JJ_GEMM_AUTO = 3
} jj_gemm;

/* What the inner solve does with a pivot block (Sec. 5.3):
 *   JJ_FULL_BLOCK      (F) the J-Jacobi method on R until its columns are
 *                      orthogonal (at most inner_max_sweeps sweeps);
 *   JJ_BLOCK_ORIENTED  (B) in the first parallel step of a sweep one sweep over
 *                      all column pairs of R, in the other steps one pass over
 *                      the off-diagonal block only (each pair (r in block i,
 *                      s in block j) annihilated once, Alg. 3.4). In the
 *                      three-level form (3B, Alg. 5.1) the same at both levels:
 *                      the first step's inner pass covers every inner block
 *                      pair, the others only the cross pairs (inner blocks of
 *                      block i against those of block j). Two-level pivots up
 *                      to 128 real columns. */
typedef enum { JJ_FULL_BLOCK = 0, JJ_BLOCK_ORIENTED = 1 } jj_block_strategy;

/* How the full-block inner solve factors a pivot A_P = R^* R (Sec. 3.3):
 *   JJ_PIVOT_CHOLESKY  the Cholesky factorization of the whole pivot (3.8);
 *   JJ_PIVOT_SPECIAL   the structure (3.7): at the start of every sweep each
 *                      block's own Gram A_ii is diagonalized (the one-sided
 *                      method on the block's columns), so that every pivot has
 *                      diagonal diagonal blocks Lambda_ii, Lambda_jj (their
 *                      off-diagonal entries, at most tol sqrt(a_rr a_ss), are
 *                      taken as zero) and R_ii = sqrt(Lambda_ii) (3.9),
 *                      R_ij = R_ii^{-1} A_ij (3.10), R_jj the Cholesky factor of
 *                      Lambda_jj - R_ij^* R_ij (3.11). Two-level full-block
 *                      solves of single problems, pivots of up to 96 complex or
 *                      128 real columns. */
typedef enum { JJ_PIVOT_CHOLESKY = 0, JJ_PIVOT_SPECIAL = 1 } jj_pivot_factor;

/* block_width value that lets the library pick the block width: at the first
 * solve of the handle, one sweep of every candidate width (powers of two from
 * 8 up to 32 for the digit forms and 64 for FP64, at most n/4) is timed on
 * a scratch copy of the input and the fastest is kept (see jj_info.block_width). */
#define JJ_BLOCK_AUTO (-1)

typedef enum {
    JJ_OK = 0,
    JJ_INVALID_ARG = 1,    /* m < n, n < 1, bad ld, J entry not +-1, bad params */
    JJ_NOT_CONVERGED = 2,  /* max_sweeps reached; results are still extractable */
    JJ_NOT_POSDEF = 3,     /* G not of full column rank in working precision
                              (a pivot Cholesky or a hyperbolic rotation failed,
                              Secs. 2.2, 3.2) */
    JJ_NONFINITE = 4,      /* NaN or Inf met in G or in a rotation */
    JJ_DEVICE_TIMEOUT = 5, /* a bounded device-side wait expired */
    JJ_CUDA_ERROR = 6,     /* a CUDA runtime call failed */
    JJ_NOT_SOLVED = 7      /* extract called before a successful solve */
} jj_status;

typedef struct {
    int64_t m;                 /* rows of G (m >= n) */
    int64_t n;                 /* columns of G */
    int32_t dtype;             /* jj_dtype */
    int32_t block_width;       /* 0: plain; >0: target columns per block (b); JJ_BLOCK_AUTO */
    int32_t inner_block_width; /* 0: two-level; >0: inner block width (three-level) */
    int32_t order;             /* jj_order (blocked form; the plain form is round-robin) */
    int32_t gemm;              /* jj_gemm */
    int32_t ozaki_slices;      /* balanced 8-bit digits per operand of the split-precision
                                  update, 1..11, 0: 11 */
    double tol;                /* <= 0: 128 * 2^-53; rotate when |a_rs| > tol sqrt(a_rr a_ss) */
    int32_t max_sweeps;        /* <= 0: 60 */
    int32_t inner_max_sweeps;  /* <= 0: 30 (inner J-Jacobi on R, blocked form) */
    void *cuda_stream;         /* cudaStream_t to run on; NULL: the legacy default stream */
    int32_t profile;           /* 1: time every kernel family of every step with CUDA events
                                  (sweeps then run without graph capture); see
                                  jjacobi_kernel_times */
    int32_t block_strategy;    /* jj_block_strategy (blocked form) */
    int32_t pivot_factor;      /* jj_pivot_factor (full-block two-level form) */
} jj_params;

typedef struct {
    int32_t status;            /* jj_status of the call */
    int32_t sweeps;            /* sweeps run (the last one applied no rotation if converged) */
    int64_t rotations;         /* rotations applied (inner rotations in the blocked form) */
    double last_max_offdiag;   /* max |a_rs| / sqrt(a_rr a_ss) seen in the last sweep */
    double seconds;            /* wall time of the call */
    int32_t block_width;       /* block width actually used (0 for plain) */
    int32_t nbl;               /* number of blocks (2 x pairs per step), 0 for plain */
    int32_t steps_per_sweep;   /* parallel steps per sweep */
    int32_t kernel_launches;   /* kernels launched by the call */
    int64_t pairs_evaluated;   /* pivot pairs whose Gram and inner solve ran (blocked form;
                                  the others were skipped as unchanged) */
    int64_t pairs_rotated;     /* pivot pairs whose inner solve applied a rotation */
} jj_info;

/* Fill *p with defaults for an m x n problem of the given dtype (plain form). */
void jjacobi_default_params(jj_params *p, int64_t m, int64_t n, int32_t dtype);

/* Create a solver handle for problems of size p->m x p->n: validates the
 * parameters, allocates every device workspace (the work copy of G, whose
 * block columns the update transforms in place (Sec. 3.3), the pivot Gram/R/W
 * blocks, the ordering tables and counters). Returns JJ_INVALID_ARG or
 * JJ_CUDA_ERROR on failure, with *h set to NULL. */
int jjacobi_create(jj_handle *h, const jj_params *p);

/* Solve H = G J G^* in place: G (device, m x n, leading dimension ldg >= m,
 * dtype of the handle) is overwritten by G~ = G W in the caller's column order
 * (the final re-permutation of Sec. 3.3). J (host, n entries of +-1) is copied.
 * Columns are permuted internally so that J = diag(I, -I) (Sec. 2.3).
 * info may be NULL; otherwise it receives the status and the elapsed seconds on
 * every return, errors included. The handle keeps the G pointer for
 * jjacobi_extract. */
int jjacobi_solve(jj_handle h, void *G, int64_t ldg, const int8_t *J, jj_info *info);

/* Eigenpairs of the last solve (Alg. 5.2): lambda[i] = J_ii ||g~_i||^2
 * (host or device pointer, n doubles, detected), and if U is not NULL
 * (device, m x n, ldu >= m, dtype of the handle) u_i = g~_i / ||g~_i||.
 * Column i belongs to column i of the caller's G. sort != 0 sorts lambda
 * ascending (and U with it). */
int jjacobi_extract(jj_handle h, double *lambda, void *U, int64_t ldu, int32_t sort);

/* End-to-end call with host buffers: copies G_host (m x n, ldg) to the device,
 * solves, extracts lambda_host (n doubles) and, if U_host is not NULL, the
 * eigenvectors (m x n, ldu), and copies them back. G_host is not modified.
 * info (may be NULL) is filled as by jjacobi_solve, with the seconds of the
 * whole call. */
int jjacobi_solve_host(jj_handle h, const void *G_host, int64_t ldg, const int8_t *J,
                       double *lambda_host, void *U_host, int64_t ldu, jj_info *info);

/* Batched solve of `count` independent problems of uneven order: the problems
 * sit side by side in one work matrix, each with its own block partition (3.3)
 * and parallel ordering (Sec. 4), and parallel step t of the batch runs step t
 * of every problem in one launch per kernel (one CUDA graph per sweep). Each
 * problem stops being transformed after its first sweep without rotations.
 * G[k] (device, m[k] x n[k], ldg[k] >= m[k], 1 <= n[k] <= m[k]) is overwritten
 * by G~_k in its own column order; J[k] (host, n[k] entries of +-1).
 * The handle's m and n bound the sizes (m[k] <= p->m, n[k] <= p->n); its
 * block_width is used for every problem (capped at ceil(n[k]/2)), or, when 0,
 * a default width (16 complex / 32 real columns for the digit forms, 32 for
 * FP64), or, for JJ_BLOCK_AUTO, the width autotuned per size class. Batched solves are two-level (inner_block_width
 * is not used). Workspaces are (re)allocated on the first call
 * and kept while the shapes repeat. lambda_out (host or device, detected; sum of
 * n[k] doubles, problem k at offset sum_{l<k} n[l], each in its own column
 * order) receives lambda_i = J_ii ||g~_i||^2 if not NULL. A problem whose blocked
 * sweeps stop on a pivot Gram block that is not positive definite in working
 * precision (columns too close to dependent for A_P = G_P^* G_P, Sec. 3.2) is
 * finished by the plain method from its current columns; its jj_info then
 * reports block_width 0. infos (may be NULL) receives one jj_info per problem
 * (pairs_evaluated, pairs_rotated, kernel_launches, seconds and
 * last_max_offdiag are batch totals); on an error before the problems' own
 * results exist (invalid arguments, a failed allocation or launch), every entry
 * carries that status and zero counts. A batch whose parallel step would hold
 * more than 65535 block pairs is refused with JJ_INVALID_ARG (split it).
 * Returns the first non-OK problem status, else JJ_OK. jjacobi_extract does
 * not apply. */
int jjacobi_solve_batched(jj_handle h, int32_t count, void *const *G, const int64_t *m,
                          const int64_t *n, const int64_t *ldg, const int8_t *const *J,
                          double *lambda_out, jj_info *infos);

/* Release the handle and every device resource it owns. NULL is a no-op. */
void jjacobi_destroy(jj_handle h);

/* Human-readable name of a jj_status value. */
const char *jjacobi_status_string(int status);

/* Device time spent by kernel family in all solves of this handle since its
 * creation, measured with CUDA events on the handle's stream when the handle
 * was created with profile = 1 (zeros otherwise). times_ms (host, 8 doubles):
 * [0] column exponents + Gram (3.6), [1] Cholesky + inner J-Jacobi (3.12),
 * [2] update (2.9), [3] plain pair steps, [4] column norms, [5..7] reserved.
 * launches (host, 8 int64, may be NULL): the matching launch counts. */
int jjacobi_kernel_times(jj_handle h, double *times_ms, int64_t *launches);

/* Front end (Sec. 2.2, (2.5)): a factor G and signs J with H = G J G^* for a
 * Hermitian H (device, n x n, column-major, ldh >= n, both triangles; the
 * dtype's element type; not modified). Symmetric Gaussian elimination with
 * complete (Bunch-Parlett) pivoting, P H P^T = M D M^*: at each step mu0 is
 * the largest modulus of the Schur complement and mu1 the largest on its
 * diagonal; a 1x1 pivot at the largest diagonal entry when
 * mu1 >= (1 + sqrt 17)/8 mu0, else the 2x2 pivot on the off-diagonal entry
 * of modulus mu0 (ties: the first entry in row-major order). Elimination stops
 * when mu0 falls to rank_tol times the largest modulus of H (rank_tol <= 0:
 * 16 n 2^-53); r is the number of eliminated columns. Each block of D is
 * diagonalized (a 2x2 block as Q diag(delta) Q^*, delta ascending), the
 * columns of M are scaled by |delta|^(1/2), and the rows are returned to H's
 * order: G (device, column-major with ldg >= n, at least n columns; the
 * first r are written) has full column rank, and J (host, n entries; the
 * first r are written) holds sign(delta). perm (host, n, may be NULL) receives P (row i of P H P^T is
 * row perm[i] of H), pivot_size (host, n, may be NULL) 1 or 2 at the first
 * column of each pivot and 0 elsewhere, rank (host) r. The zero eigenvalues
 * of a singular H (n - r of them) are not completed here. Works on the given
 * stream and synchronizes it; scratch from the stream-ordered allocator.
 * JJ_DEVICE_TIMEOUT if a grid-wide wait of the elimination ran out. */
int jjacobi_factor(int32_t dtype, const void *H, int64_t ldh, int64_t n, double rank_tol, void *G,
                   int64_t ldg, int8_t *J, int32_t *perm, int8_t *pivot_size, int64_t *rank,
                   void *stream);

/* Bound, in nanoseconds of wall-clock time, of every device-side wait in this
 * handle's tensor-core kernels (an mbarrier wait for a product, a copy or a
 * pipeline stage; the kernels' failure path for a barrier nothing arrives at).
 * A wait that runs out makes its kernel set an error flag, wait (again
 * bounded) for its own products in flight, free its tensor memory and return;
 * the solve then returns JJ_DEVICE_TIMEOUT and the handle stays usable. ns <= 0
 * restores the default of 2 s, far above any wait of a healthy run. A bound of
 * 1 ns makes every wait that does not succeed at its first poll expire: a
 * way to exercise the failure path without a fault. Not a passage of the
 * paper: a property of this implementation. */
int jjacobi_set_wait_limit(jj_handle h, int64_t ns);

/* Library version (JJACOBI_VERSION). */
int32_t jjacobi_version(void);

/* The block pairs of one sweep of the parallel ordering for nbl blocks
 * (nbl even >= 2): Initialize (Alg. 4.1) then RLStep (Alg. 4.3) or MMStep
 * (Alg. 4.2) for every process, sweep number `sweep` (>= 1). Writes
 * steps x (nbl/2) pairs (i, j), 0-based, i < j, pair q being the pivot of
 * process q, into pairs (host, capacity >= 2 * nbl * nbl/2 ints) and returns the
 * number of steps, or -1 on invalid arguments. */
int32_t jjacobi_schedule(int32_t nbl, int32_t order, int32_t sweep, int32_t *pairs);

#ifdef __cplusplus
}
#endif

#endif /* JJACOBI_H */
