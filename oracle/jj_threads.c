/* Multithreaded CPU baseline of the plain one-sided J-Jacobi method.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, like everything under oracle/: the
 * tests and the benchmark's CPU-baseline leg use it; the product library
 * neither includes, links nor calls it.
 *
 * It runs the round-robin parallel order over single columns (the modified
 * round-robin of Alg. 4.3, one column per "block") on all host cores: the
 * column pairs of one parallel step are disjoint, so they are divided among
 * the threads, and a barrier separates the steps. The per-pair arithmetic is
 * the oracle's (Alg. 3.1, from jj_oracle_body.h), so a converged solve gives
 * the same bits as the sequential oracle in round-robin order. The diagonal
 * is recomputed at the start of every sweep (Alg. 3.2); a sweep without
 * rotations ends the solve.
 */
#define _POSIX_C_SOURCE 200809L /* pthread barriers under -std=c11 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

#define R double
#define SQRT sqrt
#define FABS fabs

#define CPLX 1
#define SFX zt
#include "jj_oracle_body.h"
#undef CPLX
#undef SFX

#define CPLX 0
#define SFX dt
#include "jj_oracle_body.h"
#undef CPLX
#undef SFX

typedef struct {
    int cplx;
    int64_t m, n, ld;
    double *G;
    const int *J;
    double tol;
    int max_sweeps;
    const int *table; /* [steps][npl/2][2] column pairs, entries >= n are the dummy column */
    int steps, npl, nthreads;
    double *d;
    int64_t *rot_t;   /* per-thread rotations of the current sweep */
    double *maxoff_t; /* per-thread largest scaled off-diagonal of the current sweep */
    int *fail_t;      /* per-thread loss of positive definiteness */
    pthread_barrier_t bar;
    /* start gate: the created threads wait here until every thread exists
     * (go = 1) or a creation failed (go = -1, they return at once), so no
     * thread ever waits on a barrier that some participant will not reach */
    pthread_mutex_t gate_mu;
    pthread_cond_t gate_cv;
    int go;
    /* decided by thread 0 at the end of each sweep */
    int stop, status, sweeps;
    int64_t total;
    double maxoff;
} Team;

typedef struct {
    Team *team;
    int tid;
} Arg;

static int pair_pivot(Team *T, int64_t a, int64_t b, double *maxoff)
{
    if (T->cplx)
        return pivotzt(T->m, T->G, T->ld, NULL, 0, 0, T->J, T->d, a, b, T->tol, 0, maxoff);
    return pivotdt(T->m, T->G, T->ld, NULL, 0, 0, T->J, T->d, a, b, T->tol, 0, maxoff);
}

static double col_norm2(Team *T, int64_t i)
{
    double re, im;
    const double *g = T->G + (int64_t)(T->cplx ? 2 : 1) * i * T->ld;
    if (T->cplx)
        dotzt(T->m, g, g, &re, &im);
    else
        dotdt(T->m, g, g, &re, &im);
    return re;
}

static void *worker(void *p)
{
    Arg *A = (Arg *)p;
    Team *T = A->team;
    const int tid = A->tid, nt = T->nthreads, half = T->npl / 2;
    int sweep, go;
    pthread_mutex_lock(&T->gate_mu);
    while (T->go == 0) pthread_cond_wait(&T->gate_cv, &T->gate_mu);
    go = T->go;
    pthread_mutex_unlock(&T->gate_mu);
    if (go < 0) return NULL;
    for (sweep = 1; sweep <= T->max_sweeps; ++sweep) {
        int64_t i, rot = 0;
        double maxoff = 0;
        int fail = 0, st, q;
        for (i = tid; i < T->n; i += nt) T->d[i] = col_norm2(T, i);
        pthread_barrier_wait(&T->bar);
        for (st = 0; st < T->steps; ++st) {
            for (q = tid; q < half && !fail; q += nt) {
                int64_t a = T->table[2 * (st * half + q)];
                int64_t b = T->table[2 * (st * half + q) + 1];
                int rc;
                if (a >= T->n || b >= T->n) continue; /* dummy column */
                if (a > b) { int64_t t = a; a = b; b = t; }
                rc = pair_pivot(T, a, b, &maxoff);
                if (rc < 0) fail = 1;
                else rot += rc;
            }
            pthread_barrier_wait(&T->bar);
        }
        T->rot_t[tid] = rot;
        T->maxoff_t[tid] = maxoff;
        T->fail_t[tid] = fail;
        pthread_barrier_wait(&T->bar);
        if (tid == 0) {
            int64_t r = 0;
            double mo = 0;
            int f = 0, k;
            for (k = 0; k < nt; ++k) {
                r += T->rot_t[k];
                if (T->maxoff_t[k] > mo) mo = T->maxoff_t[k];
                f |= T->fail_t[k];
            }
            T->maxoff = mo;
            T->sweeps = sweep;
            if (f) {
                T->status = 3; /* the sequential oracle counts no rotation of this sweep */
                T->stop = 1;
            } else {
                T->total += r;
                if (r == 0) { T->status = 0; T->stop = 1; }
            }
        }
        pthread_barrier_wait(&T->bar);
        if (T->stop) break;
    }
    return NULL;
}

/* Plain J-Jacobi in round-robin order on nthreads threads.
 *   cplx   1: G is complex (interleaved re, im); 0: real.
 *   G      m x n, column-major, leading dimension ld; overwritten by G~.
 *   J      n entries, each +1 or -1.
 *   table  the round-robin sweep over single columns: steps x (npl/2) pairs,
 *          npl = n rounded up to even (column npl-1 = n is the dummy).
 * Returns 0 converged, 2 not converged after max_sweeps, 3 loss of positive
 * definiteness, 1 invalid argument or no resources. */
int jjt_solve_rr(int cplx, int64_t m, int64_t n, double *G, int64_t ld, const int *J,
                 double tol, int max_sweeps, const int *table, int steps, int nthreads,
                 int *sweeps_out, int64_t *rot_out, double *maxoff_out)
{
    Team T;
    Arg *args;
    pthread_t *th;
    int k, started = 0;
    int64_t i;
    if (m < n || n < 1 || ld < m || nthreads < 1 || max_sweeps < 1 || !table || steps < 0)
        return 1;
    for (i = 0; i < n; ++i)
        if (J[i] != 1 && J[i] != -1) return 1;
    T.cplx = cplx;
    T.m = m; T.n = n; T.ld = ld; T.G = G; T.J = J; T.tol = tol;
    T.max_sweeps = max_sweeps; T.table = table; T.steps = steps;
    T.npl = (int)(n + (n & 1)); T.nthreads = nthreads;
    T.stop = 0; T.status = 2; T.sweeps = max_sweeps; T.total = 0; T.maxoff = 0; T.go = 0;
    T.d = (double *)malloc(sizeof(double) * (size_t)n);
    T.rot_t = (int64_t *)calloc((size_t)nthreads, sizeof(int64_t));
    T.maxoff_t = (double *)calloc((size_t)nthreads, sizeof(double));
    T.fail_t = (int *)calloc((size_t)nthreads, sizeof(int));
    args = (Arg *)malloc(sizeof(Arg) * (size_t)nthreads);
    th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!T.d || !T.rot_t || !T.maxoff_t || !T.fail_t || !args || !th ||
        pthread_barrier_init(&T.bar, NULL, (unsigned)nthreads) != 0) {
        free(T.d); free(T.rot_t); free(T.maxoff_t); free(T.fail_t); free(args); free(th);
        return 1;
    }
    pthread_mutex_init(&T.gate_mu, NULL);
    pthread_cond_init(&T.gate_cv, NULL);
    for (k = 0; k < nthreads; ++k) {
        args[k].team = &T;
        args[k].tid = k;
    }
    /* threads 1..nthreads-1 are created; the caller's thread is thread 0 */
    for (k = 1; k < nthreads; ++k) {
        if (pthread_create(&th[k], NULL, worker, &args[k]) != 0) break;
        ++started;
    }
    pthread_mutex_lock(&T.gate_mu);
    T.go = started == nthreads - 1 ? 1 : -1;
    pthread_cond_broadcast(&T.gate_cv);
    pthread_mutex_unlock(&T.gate_mu);
    if (T.go > 0) worker(&args[0]);
    for (k = 1; k <= started; ++k) pthread_join(th[k], NULL);
    pthread_barrier_destroy(&T.bar);
    pthread_cond_destroy(&T.gate_cv);
    pthread_mutex_destroy(&T.gate_mu);
    free(T.d); free(T.rot_t); free(T.maxoff_t); free(T.fail_t); free(args); free(th);
    if (started != nthreads - 1) return 1;
    if (sweeps_out) *sweeps_out = T.sweeps;
    if (rot_out) *rot_out = T.total;
    if (maxoff_out) *maxoff_out = T.maxoff;
    return T.status;
}
