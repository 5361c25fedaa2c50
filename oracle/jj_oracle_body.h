/* Oracle body, instantiated by jj_oracle.c once per (real type, real/complex).
 *
 * TEST INFRASTRUCTURE ONLY: the plain CPU oracle for the one-sided hyperbolic
 * (J-)Jacobi method. Nothing in the product library includes or links this.
 *
 * Macros supplied by the includer:
 *   R      real scalar type (double or long double)
 *   CPLX   1 for complex (interleaved re,im pairs), 0 for real
 *   SFX    name suffix token
 *   SQRT, FABS  the real sqrt / fabs for R
 */

#define CAT_(a, b) a##b
#define CAT(a, b) CAT_(a, b)
#define FN(name) CAT(name, SFX)

#if CPLX
#define ESZ 2
#else
#define ESZ 1
#endif

/* Rotation parameters for one pivot pair, Alg. 3.1 (the modified rotation
 * (2.3) in the complex case), with these readings of the printed text:
 *   hyp = +J_rr * J_ss (+1: trigonometric, -1: hyperbolic);
 *   d_rr <- d_rr - hyp*t*eta, d_ss <- d_ss + t*eta;
 *   sgn(0) = +1;
 *   |theta| > 1e150: t = sgn(theta) / (2 |theta|) (first order, avoids theta^2
 *   overflow).
 * Returns 0 on success, 1 if the hyperbolic case meets theta^2 < 1 (the pivot
 * pair is not positive definite in working precision).
 *
 * `mutation` plants a deliberate mistake for the pin-sensitivity tests:
 *   1: hyp = -J_rr*J_ss as printed; 2: d_rr <- d_rr + hyp*t*eta as printed. */
static int FN(rot_params)(R arr, R ass, R ars_re, R ars_im, int hyp, int mutation,
                          R *c_out, R *s_out, R *e_re, R *e_im, R *t_out, R *eta_out,
                          R *dr_new, R *ds_new)
{
    R abs_ars, eta, theta, t, h, c, s;
    int sg;
    if (mutation == 1) hyp = -hyp;
#if CPLX
    abs_ars = SQRT(ars_re * ars_re + ars_im * ars_im);
#else
    abs_ars = FABS(ars_re);
    (void)ars_im;
#endif
    sg = (ars_re >= 0) ? 1 : -1;            /* sgn(Re a_rs), sgn(0) = +1 */
    eta = (R)sg * abs_ars;                  /* eta = sgn(Re a_rs) |a_rs| */
#if CPLX
    *e_re = ars_re / eta;                   /* e^{i alpha} = a_rs / eta */
    *e_im = ars_im / eta;
#else
    *e_re = 1;                              /* real case: eta = a_rs, no phase */
    *e_im = 0;
#endif
    theta = (R)hyp * (ass - (R)hyp * arr) / (2 * eta);
    if (FABS(theta) > (R)1e150) {
        t = (theta >= 0 ? (R)1 : (R)-1) / (2 * FABS(theta));
    } else {
        R rad = theta * theta + (R)hyp;
        if (rad < 0) return 1;
        t = (theta >= 0 ? (R)1 : (R)-1) / (FABS(theta) + SQRT(rad));
    }
    {
        R q = 1 + (R)hyp * t * t;
        if (!(q > 0)) return 1;
        h = SQRT(q);
    }
    c = 1 / h;
    s = c * t;
    *c_out = c;
    *s_out = s;
    *t_out = t;
    *eta_out = eta;
    if (mutation == 2)
        *dr_new = arr + (R)hyp * t * eta;
    else
        *dr_new = arr - (R)hyp * t * eta;
    *ds_new = ass + t * eta;
    return 0;
}

/* a = x^* y over m entries (column-major columns). */
static void FN(dot)(int64_t m, const R *x, const R *y, R *re, R *im)
{
    R sr = 0, si = 0;
    int64_t l;
    for (l = 0; l < m; ++l) {
#if CPLX
        R xr = x[2 * l], xi = x[2 * l + 1], yr = y[2 * l], yi = y[2 * l + 1];
        sr += xr * yr + xi * yi;            /* conj(x) * y */
        si += xr * yi - xi * yr;
#else
        sr += x[l] * y[l];
#endif
    }
    *re = sr;
    *im = si;
}

/* Update of the pivot columns (2.13) with the modified rotation:
 *   f = e^{i alpha} x;  x <- c f - hyp s y;  y <- s f + c y.
 * `mutation` 3 writes the second result into x as the printed text does. */
static void FN(rotate)(int64_t m, R *x, R *y, R c, R s, R e_re, R e_im, int hyp,
                       int mutation)
{
    int64_t l;
    for (l = 0; l < m; ++l) {
#if CPLX
        R fr = e_re * x[2 * l] - e_im * x[2 * l + 1];
        R fi = e_re * x[2 * l + 1] + e_im * x[2 * l];
        R yr = y[2 * l], yi = y[2 * l + 1];
        R xr_new = c * fr - (R)hyp * s * yr;
        R xi_new = c * fi - (R)hyp * s * yi;
        R yr_new = s * fr + c * yr;
        R yi_new = s * fi + c * yi;
        x[2 * l] = xr_new;
        x[2 * l + 1] = xi_new;
        if (mutation == 3) {
            x[2 * l] = yr_new;
            x[2 * l + 1] = yi_new;
        } else {
            y[2 * l] = yr_new;
            y[2 * l + 1] = yi_new;
        }
#else
        R f = e_re * x[l];
        R yv = y[l];
        R x_new = c * f - (R)hyp * s * yv;
        R y_new = s * f + c * yv;
        x[l] = x_new;
        if (mutation == 3)
            x[l] = y_new;
        else
            y[l] = y_new;
        (void)e_im;
#endif
    }
}

/* One pivot (r, s): Alg. 3.1 body. Returns 1 if a rotation was applied,
 * 0 if skipped, -1 on loss of positive definiteness. */
static int FN(pivot)(int64_t m, R *G, int64_t ld, R *W, int64_t ldw, int64_t nw,
                     const int *J, R *d, int64_t r, int64_t s, R tol, int mutation,
                     R *maxoff)
{
    R ars_re, ars_im, abs_ars, c, sn, e_re, e_im, t, eta, dr, ds, rel;
    int hyp;
    R *gr = G + (int64_t)ESZ * r * ld;
    R *gs = G + (int64_t)ESZ * s * ld;
    FN(dot)(m, gr, gs, &ars_re, &ars_im);
#if CPLX
    abs_ars = SQRT(ars_re * ars_re + ars_im * ars_im);
#else
    abs_ars = FABS(ars_re);
#endif
    rel = abs_ars / SQRT(d[r] * d[s]);
    if (rel > *maxoff) *maxoff = rel;
    if (!(rel > tol)) return 0;             /* |a_rs| <= tol sqrt(a_rr a_ss): skip */
    hyp = J[r] * J[s];
    if (FN(rot_params)(d[r], d[s], ars_re, ars_im, hyp, mutation, &c, &sn, &e_re, &e_im,
                       &t, &eta, &dr, &ds))
        return -1;
    d[r] = dr;
    d[s] = ds;
    FN(rotate)(m, gr, gs, c, sn, e_re, e_im, hyp, mutation);
    if (W)
        FN(rotate)(nw, W + (int64_t)ESZ * r * ldw, W + (int64_t)ESZ * s * ldw, c, sn, e_re,
                   e_im, hyp, mutation);
    return 1;
}

/* Plain one-sided J-Jacobi, Alg. 3.2 with Alg. 3.1 as the cycle.
 *   G     m x n, column-major, leading dimension ld (ESZ reals per entry),
 *         overwritten by G~ = G W.
 *   J     n entries, each +1 or -1.
 *   W     optional n x n (ldw) accumulator; set to I, then W <- W W_k.
 *   order 0: row-cyclic (r outer, s inner); 1: column-cyclic (s outer, r inner,
 *         as in Alg. 3.1); 2: round-robin parallel order over columns (the
 *         modified round-robin of Alg. 4.3 applied to single columns; n padded
 *         to even with a dummy column that is never rotated).
 *   The diagonal d_i = ||g_i||^2 is recomputed at the start of every sweep and
 *   tracked through the updates inside it (Alg. 3.2).
 *   Converged when a sweep applies no rotation (Sec. 5.3).
 * Returns 0 converged, 2 not converged after max_sweeps, 3 loss of positive
 * definiteness, 1 invalid argument. */
int FN(jjo_solve_)(int64_t m, int64_t n, R *G, int64_t ld, const int *J, R tol,
                   int max_sweeps, int order, R *W, int64_t ldw, int *sweeps_out,
                   int64_t *rot_out, R *maxoff_out, int mutation,
                   const int *rr_table, int rr_steps)
{
    int64_t i, r, s, total = 0;
    int sweep, status = 2;
    R *d;
    R maxoff = 0;
    if (m < n || n < 1 || ld < m) return 1;
    for (i = 0; i < n; ++i)
        if (J[i] != 1 && J[i] != -1) return 1;
    d = (R *)malloc(sizeof(R) * (size_t)n);
    if (!d) return 1;
    if (W) {
        int64_t a, b;
        for (b = 0; b < n; ++b)
            for (a = 0; a < n * ESZ; ++a) W[(int64_t)ESZ * b * ldw + a] = 0;
        for (b = 0; b < n; ++b) W[(int64_t)ESZ * b * ldw + ESZ * b] = 1;
    }
    for (sweep = 1; sweep <= max_sweeps; ++sweep) {
        int64_t rot = 0;
        maxoff = 0;
        for (i = 0; i < n; ++i) {
            R re, im;
            FN(dot)(m, G + (int64_t)ESZ * i * ld, G + (int64_t)ESZ * i * ld, &re, &im);
            d[i] = re;
        }
        if (order == 2) {
            int st, p;
            int npl = (int)(n + (n & 1));
            for (st = 0; st < rr_steps; ++st) {
                for (p = 0; p < npl / 2; ++p) {
                    int64_t a = rr_table[2 * (st * (npl / 2) + p)];
                    int64_t b = rr_table[2 * (st * (npl / 2) + p) + 1];
                    int rc;
                    if (a >= n || b >= n) continue;  /* dummy column */
                    if (a > b) { int64_t tmp = a; a = b; b = tmp; }
                    rc = FN(pivot)(m, G, ld, W, ldw, n, J, d, a, b, tol, mutation, &maxoff);
                    if (rc < 0) { status = 3; goto done; }
                    rot += rc;
                }
            }
        } else if (order == 0) {
            for (r = 0; r < n - 1; ++r)
                for (s = r + 1; s < n; ++s) {
                    int rc = FN(pivot)(m, G, ld, W, ldw, n, J, d, r, s, tol, mutation, &maxoff);
                    if (rc < 0) { status = 3; goto done; }
                    rot += rc;
                }
        } else {
            for (s = 1; s < n; ++s)
                for (r = 0; r < s; ++r) {
                    int rc = FN(pivot)(m, G, ld, W, ldw, n, J, d, r, s, tol, mutation, &maxoff);
                    if (rc < 0) { status = 3; goto done; }
                    rot += rc;
                }
        }
        total += rot;
        if (rot == 0) { status = 0; break; }
    }
done:
    if (sweeps_out) *sweeps_out = sweep > max_sweeps ? max_sweeps : sweep;
    if (rot_out) *rot_out = total;
    if (maxoff_out) *maxoff_out = maxoff;
    free(d);
    return status;
}

/* Eigenpairs from the final G~ (Alg. 5.2, last two lines; (2.10)):
 * lambda_i = J_ii ||g_i||^2 (norm recomputed), u_i = g_i / ||g_i||. U may be NULL. */
void FN(jjo_eig_)(int64_t m, int64_t n, const R *G, int64_t ld, const int *J, R *lambda,
                  R *U, int64_t ldu)
{
    int64_t i, l;
    for (i = 0; i < n; ++i) {
        const R *g = G + (int64_t)ESZ * i * ld;
        R re, im, nrm;
        FN(dot)(m, g, g, &re, &im);
        lambda[i] = (R)J[i] * re;
        if (U) {
            nrm = SQRT(re);
            for (l = 0; l < m * ESZ; ++l) U[(int64_t)ESZ * i * ldu + l] = g[l] / nrm;
        }
    }
}

/* Exposed rotation for unit tests of the closed form. */
int FN(jjo_rotation_)(R arr, R ass, R ars_re, R ars_im, int hyp, int mutation, R *out8)
{
    return FN(rot_params)(arr, ass, ars_re, ars_im, hyp, mutation, &out8[0], &out8[1],
                          &out8[2], &out8[3], &out8[4], &out8[5], &out8[6], &out8[7]);
}

#undef ESZ
#undef FN
#undef CAT
#undef CAT_
