/*
 * ORACLE body, compiled once per arithmetic type from md3c.c (REAL, SUF, R_*
 * macros are defined there).  Test infrastructure only.
 */

/*
 * Boys function F_m(T) = int_0^1 y^{2m} exp(-T y^2) dy  (paper, Appendix A)
 * for m = 0..mmax.
 *   T < 30 : every F_m from its own positive series
 *            F_m(T) = exp(-T) sum_{i>=0} (2T)^i / ((2m+1)(2m+3)...(2m+2i+1)),
 *            which follows from expanding exp(T(1-y^2)) under the integral.
 *   T >= 30: F_0 = (1/2) sqrt(pi/T) erf(sqrt T) and the upward relation
 *            F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T), obtained by integrating
 *            the definition by parts; it damps errors while 2m+1 < 2T.
 */
static void SUF(boys_all)(int mmax, REAL T, REAL* F)
{
    if (T < (REAL)30) {
        REAL e = R_EXP(-T);
        for (int m = 0; m <= mmax; ++m) {
            REAL term = (REAL)1 / (REAL)(2 * m + 1);
            REAL sum = term;
            for (int i = 1; i < 100000; ++i) {
                term *= ((REAL)2 * T) / (REAL)(2 * m + 2 * i + 1);
                sum += term;
                if (term < R_EPS * sum) break;
            }
            F[m] = e * sum;
        }
    } else {
        REAL e = R_EXP(-T);
        REAL st = R_SQRT(T);
        F[0] = (REAL)0.5 * R_SQRT(R_PI) / st * R_ERF(st);
        for (int m = 0; m < mmax; ++m)
            F[m + 1] = ((REAL)(2 * m + 1) * F[m] - e) / ((REAL)2 * T);
    }
}

/* number of Cartesian components of a shell with l quanta */
static int SUF(ncart)(int l) { return (l + 1) * (l + 2) / 2; }

/* Cartesian exponents of component idx of shell l (x desc, then y desc) */
static void SUF(cart_xyz)(int l, int idx, int* x, int* y, int* z)
{
    int i = 0;
    for (int ax = l; ax >= 0; --ax)
        for (int ay = l - ax; ay >= 0; --ay) {
            if (i == idx) {
                *x = ax;
                *y = ay;
                *z = l - ax - ay;
                return;
            }
            ++i;
        }
}

/*
 * Hermite expansion coefficients of the bra overlap distribution along one
 * axis:  x_A^i x_B^j exp(-a x_A^2 - b x_B^2) = sum_t E[i][j][t] Lambda_t,
 * Lambda_t = (d/dP_x)^t exp(-p x_P^2).
 *   E[0][0][0] = exp(-a b/p X_AB^2)
 *   E[i+1][j][t] = E[i][j][t-1]/(2p) + X_PA E[i][j][t] + (t+1) E[i][j][t+1]
 *   E[i][j+1][t] = E[i][j][t-1]/(2p) + X_PB E[i][j][t] + (t+1) E[i][j][t+1]
 * E is stored as E[(i*(lb+1)+j)*(la+lb+2)+t].
 */
static void SUF(hermite_bra)(int la, int lb, REAL a, REAL b, REAL XA, REAL XB, REAL* E)
{
    REAL p = a + b;
    REAL XP = (a * XA + b * XB) / p;
    REAL XPA = XP - XA, XPB = XP - XB, XAB = XA - XB;
    int T = la + lb + 2;
#define EIDX(i, j, t) ((((i) * (lb + 1)) + (j)) * T + (t))
    for (int k = 0; k < (la + 1) * (lb + 1) * T; ++k) E[k] = 0;
    E[EIDX(0, 0, 0)] = R_EXP(-a * b / p * XAB * XAB);
    for (int i = 0; i < la; ++i)
        for (int t = 0; t <= i + 1; ++t) {
            REAL v = XPA * E[EIDX(i, 0, t)];
            if (t > 0) v += E[EIDX(i, 0, t - 1)] / ((REAL)2 * p);
            if (t + 1 <= i) v += (REAL)(t + 1) * E[EIDX(i, 0, t + 1)];
            E[EIDX(i + 1, 0, t)] = v;
        }
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j < lb; ++j)
            for (int t = 0; t <= i + j + 1; ++t) {
                REAL v = XPB * E[EIDX(i, j, t)];
                if (t > 0) v += E[EIDX(i, j, t - 1)] / ((REAL)2 * p);
                if (t + 1 <= i + j) v += (REAL)(t + 1) * E[EIDX(i, j, t + 1)];
                E[EIDX(i, j + 1, t)] = v;
            }
#undef EIDX
}

/*
 * One-centre Hermite coefficients of x_C^k exp(-q x_C^2):
 *   E[0][0] = 1,  E[k+1][t] = E[k][t-1]/(2q) + (t+1) E[k][t+1]
 * stored as E[k*(lc+2)+t].
 */
static void SUF(hermite_ket)(int lc, REAL q, REAL* E)
{
    int T = lc + 2;
    for (int k = 0; k < (lc + 1) * T; ++k) E[k] = 0;
    E[0] = 1;
    for (int k = 0; k < lc; ++k)
        for (int t = 0; t <= k + 1; ++t) {
            REAL v = 0;
            if (t > 0) v += E[k * T + t - 1] / ((REAL)2 * q);
            if (t + 1 <= k) v += (REAL)(t + 1) * E[k * T + t + 1];
            E[(k + 1) * T + t] = v;
        }
}

/*
 * Hermite Coulomb integrals R_{tuv} = R^{0}_{tuv}(alpha, X, Y, Z) for
 * t+u+v <= L:
 *   R^{n}_{000} = (-2 alpha)^n F_n(alpha (X^2+Y^2+Z^2))
 *   R^{n}_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X R^{n+1}_{t,u,v}   (same for u, v)
 * Full table Rn[n][t][u][v] with dimension (L+1)^4; R0 receives n = 0.
 */
static void SUF(hermite_coulomb)(int L, REAL alpha, REAL X, REAL Y, REAL Z, REAL* Rn, REAL* R0)
{
    int D = L + 1;
#define RI(n, t, u, v) ((((n) * D + (t)) * D + (u)) * D + (v))
    REAL F[ORACLE_NMAX + 1];
    SUF(boys_all)(L, alpha * (X * X + Y * Y + Z * Z), F);
    REAL f = 1;
    for (int n = 0; n <= L; ++n) {
        Rn[RI(n, 0, 0, 0)] = f * F[n];
        f *= (REAL)-2 * alpha;
    }
    /* build by increasing total order s = t+u+v, for every n <= L-s */
    for (int s = 1; s <= L; ++s)
        for (int n = 0; n <= L - s; ++n)
            for (int t = 0; t <= s; ++t)
                for (int u = 0; u <= s - t; ++u) {
                    int v = s - t - u;
                    REAL r;
                    if (t > 0) {
                        r = X * Rn[RI(n + 1, t - 1, u, v)];
                        if (t > 1) r += (REAL)(t - 1) * Rn[RI(n + 1, t - 2, u, v)];
                    } else if (u > 0) {
                        r = Y * Rn[RI(n + 1, t, u - 1, v)];
                        if (u > 1) r += (REAL)(u - 1) * Rn[RI(n + 1, t, u - 2, v)];
                    } else {
                        r = Z * Rn[RI(n + 1, t, u, v - 1)];
                        if (v > 1) r += (REAL)(v - 1) * Rn[RI(n + 1, t, u, v - 2)];
                    }
                    Rn[RI(n, t, u, v)] = r;
                }
    for (int t = 0; t <= L; ++t)
        for (int u = 0; u <= L - t; ++u)
            for (int v = 0; v <= L - t - u; ++v) R0[(t * D + u) * D + v] = Rn[RI(0, t, u, v)];
#undef RI
}

/*
 * Contracted Cartesian block (a b|c) for one shell triple, written to
 * out[ia][ib][ic] (row-major, Cartesian order as above).
 */
static int SUF(eri3c_shell)(int la, int ka, const double* A, const double* ea, const double* ca,
                            int lb, int kb, const double* B, const double* eb, const double* cb,
                            int lc, int kc, const double* C, const double* ec, const double* cc,
                            double* out)
{
    int na = SUF(ncart)(la), nb = SUF(ncart)(lb), nc = SUF(ncart)(lc);
    int Lab = la + lb, L = la + lb + lc;
    int D = L + 1;
    int TE = la + lb + 2, TK = lc + 2;
    REAL* acc = (REAL*)calloc((size_t)na * nb * nc, sizeof(REAL));
    REAL* Ex = (REAL*)malloc(sizeof(REAL) * (la + 1) * (lb + 1) * TE);
    REAL* Ey = (REAL*)malloc(sizeof(REAL) * (la + 1) * (lb + 1) * TE);
    REAL* Ez = (REAL*)malloc(sizeof(REAL) * (la + 1) * (lb + 1) * TE);
    REAL* Ek = (REAL*)malloc(sizeof(REAL) * (lc + 1) * TK);
    REAL* Rn = (REAL*)malloc(sizeof(REAL) * D * D * D * D);
    REAL* R0 = (REAL*)malloc(sizeof(REAL) * D * D * D);
    /* S[t][u][v][ic] = sum_{tau,nu,phi} (-1)^{tau+nu+phi} Ek.. R_{t+tau,u+nu,v+phi} */
    int DS = Lab + 1;
    REAL* S = (REAL*)malloc(sizeof(REAL) * DS * DS * DS * nc);
    if (!acc || !Ex || !Ey || !Ez || !Ek || !Rn || !R0 || !S) {
        free(acc); free(Ex); free(Ey); free(Ez); free(Ek); free(Rn); free(R0); free(S);
        return -2;
    }
    const REAL pi = R_PI;
    for (int ia = 0; ia < ka; ++ia)
        for (int ib = 0; ib < kb; ++ib) {
            REAL a = ea[ia], b = eb[ib], p = a + b;
            REAL P[3];
            for (int d = 0; d < 3; ++d) P[d] = (a * (REAL)A[d] + b * (REAL)B[d]) / p;
            SUF(hermite_bra)(la, lb, a, b, A[0], B[0], Ex);
            SUF(hermite_bra)(la, lb, a, b, A[1], B[1], Ey);
            SUF(hermite_bra)(la, lb, a, b, A[2], B[2], Ez);
            for (int ic = 0; ic < kc; ++ic) {
                REAL q = ec[ic];
                REAL alpha = p * q / (p + q);
                REAL pref = (REAL)2 * pi * pi * R_SQRT(pi) / (p * q * R_SQRT(p + q));
                REAL coef = (REAL)ca[ia] * (REAL)cb[ib] * (REAL)cc[ic] * pref;
                SUF(hermite_ket)(lc, q, Ek);
                SUF(hermite_coulomb)(L, alpha, P[0] - C[0], P[1] - C[1], P[2] - C[2], Rn, R0);
                for (int t = 0; t <= Lab; ++t)
                    for (int u = 0; u <= Lab - t; ++u)
                        for (int v = 0; v <= Lab - t - u; ++v)
                            for (int k = 0; k < nc; ++k) {
                                int cx, cy, cz;
                                SUF(cart_xyz)(lc, k, &cx, &cy, &cz);
                                REAL s = 0;
                                for (int tau = 0; tau <= cx; ++tau)
                                    for (int nu = 0; nu <= cy; ++nu)
                                        for (int ph = 0; ph <= cz; ++ph) {
                                            REAL e = Ek[cx * TK + tau] * Ek[cy * TK + nu] * Ek[cz * TK + ph];
                                            if (e == 0) continue;
                                            REAL sg = ((tau + nu + ph) & 1) ? (REAL)-1 : (REAL)1;
                                            s += sg * e * R0[((t + tau) * D + (u + nu)) * D + (v + ph)];
                                        }
                                S[((t * DS + u) * DS + v) * nc + k] = s;
                            }
                for (int i = 0; i < na; ++i) {
                    int ax, ay, az;
                    SUF(cart_xyz)(la, i, &ax, &ay, &az);
                    for (int j = 0; j < nb; ++j) {
                        int bx, by, bz;
                        SUF(cart_xyz)(lb, j, &bx, &by, &bz);
                        const REAL* ex = Ex + (ax * (lb + 1) + bx) * TE;
                        const REAL* ey = Ey + (ay * (lb + 1) + by) * TE;
                        const REAL* ez = Ez + (az * (lb + 1) + bz) * TE;
                        for (int k = 0; k < nc; ++k) {
                            REAL s = 0;
                            for (int t = 0; t <= ax + bx; ++t)
                                for (int u = 0; u <= ay + by; ++u)
                                    for (int v = 0; v <= az + bz; ++v)
                                        s += ex[t] * ey[u] * ez[v] * S[((t * DS + u) * DS + v) * nc + k];
                            acc[(i * nb + j) * nc + k] += coef * s;
                        }
                    }
                }
            }
        }
    for (int k = 0; k < na * nb * nc; ++k) out[k] = (double)acc[k];
    free(acc); free(Ex); free(Ey); free(Ez); free(Ek); free(Rn); free(R0); free(S);
    return 0;
}
