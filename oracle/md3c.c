/*
 * ORACLE (test infrastructure only).  Plain, slow McMurchie-Davidson
 * evaluation of contracted 3-center Coulomb integrals (ab|c) over
 * non-normalised Cartesian Gaussians.  Only tests/, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code; the GPU library never
 * does, and this file shares no code with it.
 *
 * What it computes (paper, Appendix A, definitions of the primitive
 * Cartesian Gaussian, gamma, rho, P, AB, PC and the Boys function F_m):
 *
 *   (a b|c) = sum_{primitives} c_a c_b c_c  [a b|c],
 *   [a b|c] = int int phi_a(r1) phi_b(r1) |r1-r2|^-1 phi_c(r2) dr1 dr2,
 *   phi_a(r) = (x-Ax)^ax (y-Ay)^ay (z-Az)^az exp(-zeta_a |r-A|^2).
 *
 * Scheme: McMurchie-Davidson Hermite expansion (the scheme the paper
 * considered and set aside for its GPU kernels, Sec. 2.3), i.e. a different
 * route from the Obara-Saika/HGPA recurrences (Sec. 2.5) that the GPU path
 * implements:
 *
 *   [a b|c] = 2 pi^{5/2} / (p q sqrt(p+q))
 *             sum_{tuv} E^{ab}_{tuv} sum_{tau nu phi} (-1)^{tau+nu+phi}
 *                       E^{c}_{tau nu phi} R_{t+tau,u+nu,v+phi}(alpha, P-C)
 *
 * with p = zeta_a + zeta_b (the paper's gamma), q = zeta_c,
 * alpha = p q/(p+q) (the paper's rho), E^{ab} the Hermite coefficients of the
 * bra overlap distribution (E^{00}_0 = exp(-zeta_a zeta_b/p AB^2)), E^{c} the
 * one-centre Hermite coefficients of the ket Gaussian, and R the Hermite
 * Coulomb integrals built from R^{n}_{000} = (-2 alpha)^n F_n(alpha |PC|^2).
 * The ket stays Cartesian here (a true Cartesian integral); the solid-harmonic
 * transforms are applied afterwards by oracle/solid.py.
 *
 * Two arithmetic types: double, and long double (80-bit on x86_64, binary128
 * on aarch64) used to bound the double oracle's own rounding error.
 *
 * Cartesian order inside a shell: x descending, then y descending
 * (xx, xy, xz, yy, yz, zz).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define ORACLE_LMAX_SHELL 8              /* per-shell angular momentum limit  */
#define ORACLE_NMAX (3 * ORACLE_LMAX_SHELL + 1) /* Boys orders 0..3*8 */

/* ------------------------------------------------------------------------ */
/* The body below is written once and compiled twice: REAL = double and     */
/* REAL = long double.  SUF(x) decorates function names.                    */
/* ------------------------------------------------------------------------ */

#define REAL double
#define SUF(x) x##_d
#define R_EXP exp
#define R_SQRT sqrt
#define R_ERF erf
#define R_FABS fabs
#define R_PI 3.14159265358979323846264338327950288
#define R_EPS 1.0e-17
#include "md3c_body.h"
#undef REAL
#undef SUF
#undef R_EXP
#undef R_SQRT
#undef R_ERF
#undef R_FABS
#undef R_PI
#undef R_EPS

#define REAL long double
#define SUF(x) x##_ld
#define R_EXP expl
#define R_SQRT sqrtl
#define R_ERF erfl
#define R_FABS fabsl
#define R_PI 3.14159265358979323846264338327950288L
#define R_EPS 1.0e-36L
#include "md3c_body.h"

/* ------------------------------------------------------------------------ */
/* Exported entry points (ctypes).                                          */
/* ------------------------------------------------------------------------ */

/* Boys function F_m(T) for m = 0..mmax, written to out[0..mmax]. */
void oracle_boys(int mmax, double T, int extended, double* out)
{
    if (mmax < 0 || mmax >= 64) return;
    if (extended) {
        long double tmp[64];
        boys_all_ld(mmax, (long double)T, tmp);
        for (int m = 0; m <= mmax; ++m) out[m] = (double)tmp[m];
    } else {
        boys_all_d(mmax, T, out);
    }
}

/*
 * Cartesian contracted integrals for a list of shell triples.
 *   shell tables (one combined table for all shells):
 *     sh_l[s], sh_k[s] (number of primitives), sh_off[s] (offset into prim
 *     arrays), sh_xyz[3*s], prim_exp[], prim_coef[]
 *   trip[3*i+0..2]: shell indices (a, b, c) of triple i
 *   out_off[i]: offset of triple i's block in out; the block is
 *     [nc(la)][nc(lb)][nc(lc)] row-major.
 * Returns 0 on success, -1 on invalid input.
 */
int oracle_eri3c_cart(const int32_t* sh_l, const int32_t* sh_k, const int64_t* sh_off,
                      const double* sh_xyz, const double* prim_exp, const double* prim_coef,
                      int64_t ntrip, const int32_t* trip, const int64_t* out_off,
                      double* out, int extended)
{
    for (int64_t i = 0; i < ntrip; ++i)
        for (int j = 0; j < 3; ++j)
            if (sh_l[trip[3 * i + j]] < 0 || sh_l[trip[3 * i + j]] > ORACLE_LMAX_SHELL) return -1;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < ntrip; ++i) {
        int sa = trip[3 * i], sb = trip[3 * i + 1], sc = trip[3 * i + 2];
        int rc;
        if (extended)
            rc = eri3c_shell_ld(sh_l[sa], sh_k[sa], sh_xyz + 3 * sa, prim_exp + sh_off[sa], prim_coef + sh_off[sa],
                                sh_l[sb], sh_k[sb], sh_xyz + 3 * sb, prim_exp + sh_off[sb], prim_coef + sh_off[sb],
                                sh_l[sc], sh_k[sc], sh_xyz + 3 * sc, prim_exp + sh_off[sc], prim_coef + sh_off[sc],
                                out + out_off[i]);
        else
            rc = eri3c_shell_d(sh_l[sa], sh_k[sa], sh_xyz + 3 * sa, prim_exp + sh_off[sa], prim_coef + sh_off[sa],
                               sh_l[sb], sh_k[sb], sh_xyz + 3 * sb, prim_exp + sh_off[sb], prim_coef + sh_off[sb],
                               sh_l[sc], sh_k[sc], sh_xyz + 3 * sc, prim_exp + sh_off[sc], prim_coef + sh_off[sc],
                               out + out_off[i]);
        if (rc) {
#pragma omp atomic write
            err = rc;
        }
    }
    return err;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
