/*
 * ORACLE (test infrastructure only).  Plain, slow McMurchie-Davidson
 * evaluation of contracted 3-center Coulomb integrals (ab|c) over
 * non-normalised Gaussians.  Only tests/, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code; the GPU library never
 * does, and this file shares no code with it.
 *
 * What it computes (paper, Appendix A: definitions of the primitive
 * Cartesian Gaussian, gamma, rho, P, AB, PC and the Boys function F_m; the ket
 * is a real solid-harmonic Gaussian, Sec. 2.2 / 2.5.1):
 *
 *   (a b|C) = sum_{primitives} c_a c_b c_c  [a b|C],
 *   [a b|C] = int int phi_a(r1) phi_b(r1) |r1-r2|^-1 chi_C(r2) dr1 dr2,
 *   phi_a(r) = (x-Ax)^ax (y-Ay)^ay (z-Az)^az exp(-zeta_a |r-A|^2),
 *   chi_C(r) = S_{lc,m}(r-C) exp(-zeta_c |r-C|^2)  (or a Cartesian ket).
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
 * Hermite coefficients of the ket, and R the Hermite Coulomb integrals built
 * from R^{n}_{000} = (-2 alpha)^n F_n(alpha |PC|^2).  A solid-harmonic ket is
 * expanded exactly by Hobson's theorem (see ket_terms); a solid-harmonic bra
 * is obtained by projecting the Cartesian bra in working precision.
 *
 * Three arithmetic types: double; long double (80-bit on x86_64, binary128 on
 * aarch64); and binary128 (__float128 with libquadmath on x86_64, long double
 * on aarch64).  The binary128 mode is the arbiter when the double mode loses
 * digits to cancellation in the bra projection.
 *
 * Cartesian order inside a shell: x descending, then y descending
 * (xx, xy, xz, yy, yz, zz).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define ORACLE_LMAX_SHELL 9              /* per-shell angular momentum limit  */
#define ORACLE_NMAX (3 * ORACLE_LMAX_SHELL + 3) /* Boys orders */

/* ------------------------------------------------------------------------ */
/* The body is written once and compiled per arithmetic type: REAL, and     */
/* SUF(x) decorating function names.                                        */
/* ------------------------------------------------------------------------ */

#define REAL double
#define SUF(x) x##_d
#define R_EXP exp
#define R_SQRT sqrt
#define R_ERF erf
#define R_PI 3.14159265358979323846264338327950288
#define R_EPS 1.0e-17
#include "md3c_body.h"
#undef REAL
#undef SUF
#undef R_EXP
#undef R_SQRT
#undef R_ERF
#undef R_PI
#undef R_EPS

#define REAL long double
#define SUF(x) x##_ld
#define R_EXP expl
#define R_SQRT sqrtl
#define R_ERF erfl
#define R_PI 3.14159265358979323846264338327950288L
#define R_EPS 1.0e-36L
#include "md3c_body.h"
#undef REAL
#undef SUF
#undef R_EXP
#undef R_SQRT
#undef R_ERF
#undef R_PI
#undef R_EPS

#if defined(__x86_64__)
#include <quadmath.h>
typedef __float128 quad_t_;
#define R_EXP expq
#define R_SQRT sqrtq
#define R_ERF erfq
#define R_PI M_PIq
#define R_EPS 1.0e-36Q
#else
typedef long double quad_t_;
#define R_EXP expl
#define R_SQRT sqrtl
#define R_ERF erfl
#define R_PI 3.14159265358979323846264338327950288L
#define R_EPS 1.0e-36L
#endif
#define REAL quad_t_
#define SUF(x) x##_q
#include "md3c_body.h"
#undef REAL
#undef SUF

/* ------------------------------------------------------------------------ */
/* Exported entry points (ctypes).                                          */
/* ------------------------------------------------------------------------ */

/* Boys function F_m(T) for m = 0..mmax, written to out[0..mmax];
 * mode 0 double, 1 long double, 2 binary128. */
void oracle_boys(int mmax, double T, int mode, double* out)
{
    if (mmax < 0 || mmax > ORACLE_NMAX) return;
    if (mode == 1) {
        long double tmp[ORACLE_NMAX + 1];
        boys_all_ld(mmax, (long double)T, tmp);
        for (int m = 0; m <= mmax; ++m) out[m] = (double)tmp[m];
    } else if (mode == 2) {
        quad_t_ tmp[ORACLE_NMAX + 1];
        boys_all_q(mmax, (quad_t_)T, tmp);
        for (int m = 0; m <= mmax; ++m) out[m] = (double)tmp[m];
    } else {
        boys_all_d(mmax, T, out);
    }
}

/*
 * Contracted blocks for a list of shell triples.
 *   shell tables (one combined table for all shells):
 *     sh_l[s], sh_k[s] (number of primitives), sh_off[s] (offset into prim
 *     arrays), sh_xyz[3*s], prim_exp[], prim_coef[]
 *   trip[3*i+0..2]: shell indices (a, b, c) of triple i
 *   out_off[i]: offset of triple i's block [nA][nB][nC] in out
 *   mode: 0 double, 1 long double, 2 binary128
 *   bra_pure / ket_pure: solid-harmonic bra / ket
 *   dA, dB, dC: -1 or the axis of a first derivative with respect to that centre
 *   sph_hi, sph_lo, sph_off: solid-harmonic matrices for l = 0..nsph-1 as
 *     double pairs (value = hi + lo), matrix l starting at sph_off[l]
 * Returns 0 on success, -1 on invalid input, -2 on allocation failure.
 */
int oracle_eri3c(const int32_t* sh_l, const int32_t* sh_k, const int64_t* sh_off,
                 const double* sh_xyz, const double* prim_exp, const double* prim_coef,
                 int64_t ntrip, const int32_t* trip, const int64_t* out_off, double* out,
                 int mode, int bra_pure, int ket_pure, int dA, int dB, int dC,
                 int nsph, const double* sph_hi, const double* sph_lo, const int64_t* sph_off)
{
    for (int64_t i = 0; i < ntrip; ++i)
        for (int j = 0; j < 3; ++j) {
            int l = sh_l[trip[3 * i + j]];
            if (l < 0 || l > ORACLE_LMAX_SHELL - 1) return -1;
            if ((bra_pure || ket_pure) && l >= nsph) return -1;
        }
    int64_t ntot = nsph > 0 ? sph_off[nsph] : 0;
    double* Td = (double*)malloc(sizeof(double) * (ntot + 1));
    long double* Tl = (long double*)malloc(sizeof(long double) * (ntot + 1));
    quad_t_* Tq = (quad_t_*)malloc(sizeof(quad_t_) * (ntot + 1));
    if (!Td || !Tl || !Tq) { free(Td); free(Tl); free(Tq); return -2; }
    for (int64_t k = 0; k < ntot; ++k) {
        Td[k] = sph_hi[k] + sph_lo[k];
        Tl[k] = (long double)sph_hi[k] + (long double)sph_lo[k];
        Tq[k] = (quad_t_)sph_hi[k] + (quad_t_)sph_lo[k];
    }
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < ntrip; ++i) {
        int sa = trip[3 * i], sb = trip[3 * i + 1], sc = trip[3 * i + 2];
        int rc;
#define ARGS sh_l[sa], sh_k[sa], sh_xyz + 3 * sa, prim_exp + sh_off[sa], prim_coef + sh_off[sa], \
             sh_l[sb], sh_k[sb], sh_xyz + 3 * sb, prim_exp + sh_off[sb], prim_coef + sh_off[sb], \
             sh_l[sc], sh_k[sc], sh_xyz + 3 * sc, prim_exp + sh_off[sc], prim_coef + sh_off[sc], \
             bra_pure, ket_pure, dA, dB, dC
        if (mode == 2)
            rc = eri3c_shell_q(ARGS, Tq, sph_off, out + out_off[i]);
        else if (mode == 1)
            rc = eri3c_shell_ld(ARGS, Tl, sph_off, out + out_off[i]);
        else
            rc = eri3c_shell_d(ARGS, Td, sph_off, out + out_off[i]);
#undef ARGS
        if (rc) {
#pragma omp atomic write
            err = rc;
        }
    }
    free(Td); free(Tl); free(Tq);
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
