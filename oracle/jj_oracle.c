/* CPU oracle for the one-sided hyperbolic (J-)Jacobi method.
 *
 * TEST INFRASTRUCTURE ONLY. This file, and everything under oracle/, may be
 * used by the tests, by the smoke check and by the benchmark's CPU-baseline
 * leg; the product library neither includes, links nor calls it, and it
 * shares no code with the CUDA path.
 *
 * It is the plain, non-blocked algorithm of the paper: Alg. 3.2 (repeat
 * sweeps, recompute the diagonal at each sweep) with Alg. 3.1 as the sweep,
 * in row-cyclic, column-cyclic or round-robin order, in float64 and in long
 * double, real and complex. The eigenpairs are read off as in the last lines
 * of Alg. 5.2. See jj_oracle_body.h for the readings of the printed formulas.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define R double
#define SQRT sqrt
#define FABS fabs

#define CPLX 1
#define SFX z
#include "jj_oracle_body.h"
#undef CPLX
#undef SFX

#define CPLX 0
#define SFX d
#include "jj_oracle_body.h"
#undef CPLX
#undef SFX

#undef R
#undef SQRT
#undef FABS

#define R long double
#define SQRT sqrtl
#define FABS fabsl

#define CPLX 1
#define SFX zl
#include "jj_oracle_body.h"
#undef CPLX
#undef SFX

#define CPLX 0
#define SFX dl
#include "jj_oracle_body.h"
#undef CPLX
#undef SFX

int jjo_long_double_mantissa_bits(void) { return (int)__LDBL_MANT_DIG__; }
