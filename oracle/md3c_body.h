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
static int SUF(ncart)(int l) { return l < 0 ? 0 : (l + 1) * (l + 2) / 2; }

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

static int SUF(cart_idx)(int x, int y, int z)
{
    int l = x + y + z, idx = 0;
    for (int ax = l; ax > x; --ax) idx += l - ax + 1;
    return idx + (l - x) - y;
}

/*
 * Hermite expansion coefficients of the bra overlap distribution along one
 * axis:  x_A^i x_B^j exp(-a x_A^2 - b x_B^2) = sum_t E[i][j][t] Lambda_t,
 * Lambda_t = (d/dP_x)^t exp(-p x_P^2).
 *   E[0][0][0] = exp(-a b/p X_AB^2)
 *   E[i+1][j][t] = E[i][j][t-1]/(2p) + X_PA E[i][j][t] + (t+1) E[i][j][t+1]
 *   E[i][j+1][t] = E[i][j][t-1]/(2p) + X_PB E[i][j][t] + (t+1) E[i][j][t+1]
 * E is stored as E[(i*(lb+1)+j)*(la+lb+2)+t], i <= la, j <= lb.
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
 * One-centre Hermite coefficients of x_C^k exp(-q x_C^2) (true Cartesian ket):
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
 * Ket Hermite coefficients for one ket function, as a list of
 * (tau, nu, phi, coefficient).  Returns the number of entries.
 *
 * ket_pure = 0: true Cartesian x^cx y^cy z^cz exp(-q r_C^2) (component kc).
 * ket_pure = 1: real solid harmonic S_{lc,m}(r_C) exp(-q r_C^2) (m index kc)
 *   through Hobson's theorem: for a harmonic homogeneous polynomial S of
 *   degree l, S(grad_C) exp(-q|r-C|^2) = (2q)^l S(r-C) exp(-q|r-C|^2), so the
 *   solid-harmonic Gaussian is exactly (2q)^{-l} sum_c T[m][c] Lambda_c with
 *   Hermite Gaussians Lambda_c = d^c/dC^c exp(-q|r-C|^2) of total order l only.
 *   Projecting Cartesian kets instead would form, and then cancel, their
 *   lower-order (r^2-type) parts, which for a compact ket far from the bra
 *   exceed the result by many orders of magnitude.
 * dC = -1 or an axis: the function is differentiated with respect to C_dC,
 *   d/dC_i Lambda_c = Lambda_{c+1_i} (pure), and for the Cartesian ket
 *   d/dC_i [x_C^c ..] = 2q [x_C^{c+1_i} ..] - c_i [x_C^{c-1_i} ..].
 * Tket: solid-harmonic matrix of shell lc in REAL (pure case only).
 */
static int SUF(ket_terms)(int lc, int kc, REAL q, int ket_pure, int dC, const REAL* Tket, int* tnp, REAL* coef)
{
    int n = 0;
    if (ket_pure) {
        REAL s = 1;
        for (int k = 0; k < lc; ++k) s /= (REAL)2 * q;
        int nc = SUF(ncart)(lc);
        for (int c = 0; c < nc; ++c) {
            REAL t = Tket[kc * nc + c];
            if (t == 0) continue;
            int x, y, z;
            SUF(cart_xyz)(lc, c, &x, &y, &z);
            if (dC == 0) ++x;
            if (dC == 1) ++y;
            if (dC == 2) ++z;
            tnp[3 * n] = x;
            tnp[3 * n + 1] = y;
            tnp[3 * n + 2] = z;
            coef[n++] = s * t;
        }
        return n;
    }
    /* Cartesian ket: product of one-centre expansions per axis */
    int cx, cy, cz;
    SUF(cart_xyz)(lc, kc, &cx, &cy, &cz);
    int TK = lc + 3;
    REAL Ek[(ORACLE_LMAX_SHELL + 2) * (ORACLE_LMAX_SHELL + 3)];
    SUF(hermite_ket)(lc + 1, q, Ek);
    REAL ex[ORACLE_LMAX_SHELL + 3], ey[ORACLE_LMAX_SHELL + 3], ez[ORACLE_LMAX_SHELL + 3];
    int c3[3] = {cx, cy, cz};
    REAL* e3[3] = {ex, ey, ez};
    for (int d = 0; d < 3; ++d) {
        for (int t = 0; t < TK; ++t) e3[d][t] = 0;
        if (d == dC) {
            for (int t = 0; t <= c3[d] + 1; ++t) {
                REAL v = (REAL)2 * q * Ek[(c3[d] + 1) * TK + t];
                if (c3[d] > 0) v -= (REAL)c3[d] * Ek[(c3[d] - 1) * TK + t];
                e3[d][t] = v;
            }
        } else {
            for (int t = 0; t <= c3[d]; ++t) e3[d][t] = Ek[c3[d] * TK + t];
        }
    }
    for (int t = 0; t < TK; ++t)
        for (int u = 0; u < TK; ++u)
            for (int v = 0; v < TK; ++v) {
                REAL e = ex[t] * ey[u] * ez[v];
                if (e == 0) continue;
                tnp[3 * n] = t;
                tnp[3 * n + 1] = u;
                tnp[3 * n + 2] = v;
                coef[n++] = e;
            }
    return n;
}

/*
 * Contracted block for one shell triple, written (as double) to out:
 *   [nA][nB][nC] with nA = bra_pure ? 2la+1 : ncart(la) (same for B) and
 *   nC = ket_pure ? 2lc+1 : ncart(lc).
 * dA, dB, dC: -1, or the axis of a derivative with respect to that centre
 * (d/dA_i phi_a = 2 zeta_a phi_{a+1_i} - a_i phi_{a-1_i}, from differentiating
 * the definition in Appendix A).  The bra is expanded in Cartesian form and
 * projected onto solid harmonics at the end, in working precision.
 * Tsph: solid-harmonic matrices in working precision; Tsph + Toff[l].
 */
static int SUF(eri3c_shell)(int la, int ka, const double* A, const double* ea, const double* ca,
                            int lb, int kb, const double* B, const double* eb, const double* cb,
                            int lc, int kc, const double* C, const double* ec, const double* cc,
                            int bra_pure, int ket_pure, int dA, int dB, int dC,
                            const REAL* Tsph, const int64_t* Toff, double* out)
{
    int na = SUF(ncart)(la), nb = SUF(ncart)(lb), nkc = ket_pure ? 2 * lc + 1 : SUF(ncart)(lc);
    int la1 = la + (dA >= 0), lb1 = lb + (dB >= 0);
    int Lab = la1 + lb1, L = Lab + lc + (dC >= 0);
    int D = L + 1;
    int TE = la1 + lb1 + 2;
    int DS = Lab + 1;
    REAL* acc = (REAL*)calloc((size_t)na * nb * nkc, sizeof(REAL));
    REAL* Ex = (REAL*)malloc(sizeof(REAL) * (la1 + 1) * (lb1 + 1) * TE);
    REAL* Ey = (REAL*)malloc(sizeof(REAL) * (la1 + 1) * (lb1 + 1) * TE);
    REAL* Ez = (REAL*)malloc(sizeof(REAL) * (la1 + 1) * (lb1 + 1) * TE);
    REAL* Rn = (REAL*)malloc(sizeof(REAL) * D * D * D * D);
    REAL* R0 = (REAL*)malloc(sizeof(REAL) * D * D * D);
    REAL* S = (REAL*)malloc(sizeof(REAL) * DS * DS * DS * nkc);
    int maxk = 1000;
    int* ktnp = (int*)malloc(sizeof(int) * 3 * maxk);
    REAL* kcoef = (REAL*)malloc(sizeof(REAL) * maxk);
    REAL* bx = (REAL*)malloc(sizeof(REAL) * TE);
    REAL* by = (REAL*)malloc(sizeof(REAL) * TE);
    REAL* bz = (REAL*)malloc(sizeof(REAL) * TE);
    if (!acc || !Ex || !Ey || !Ez || !Rn || !R0 || !S || !ktnp || !kcoef || !bx || !by || !bz) {
        free(acc); free(Ex); free(Ey); free(Ez); free(Rn); free(R0); free(S); free(ktnp); free(kcoef);
        free(bx); free(by); free(bz);
        return -2;
    }
    const REAL pi = R_PI;
    const REAL* Tket = ket_pure ? Tsph + Toff[lc] : 0;
#define EI(E, i, j, t) (E)[(((i) * (lb1 + 1)) + (j)) * TE + (t)]
    for (int ia = 0; ia < ka; ++ia)
        for (int ib = 0; ib < kb; ++ib) {
            REAL a = ea[ia], b = eb[ib], p = a + b;
            REAL P[3];
            for (int d = 0; d < 3; ++d) P[d] = (a * (REAL)A[d] + b * (REAL)B[d]) / p;
            SUF(hermite_bra)(la1, lb1, a, b, A[0], B[0], Ex);
            SUF(hermite_bra)(la1, lb1, a, b, A[1], B[1], Ey);
            SUF(hermite_bra)(la1, lb1, a, b, A[2], B[2], Ez);
            for (int ic = 0; ic < kc; ++ic) {
                REAL q = ec[ic];
                REAL alpha = p * q / (p + q);
                REAL pref = (REAL)2 * pi * pi * R_SQRT(pi) / (p * q * R_SQRT(p + q));
                REAL coef = (REAL)ca[ia] * (REAL)cb[ib] * (REAL)cc[ic] * pref;
                SUF(hermite_coulomb)(L, alpha, P[0] - C[0], P[1] - C[1], P[2] - C[2], Rn, R0);
                for (int k = 0; k < nkc; ++k) {
                    int nt = SUF(ket_terms)(lc, k, q, ket_pure, dC, Tket, ktnp, kcoef);
                    for (int t = 0; t <= Lab; ++t)
                        for (int u = 0; u <= Lab - t; ++u)
                            for (int v = 0; v <= Lab - t - u; ++v) {
                                REAL s = 0;
                                for (int j = 0; j < nt; ++j) {
                                    int tau = ktnp[3 * j], nu = ktnp[3 * j + 1], ph = ktnp[3 * j + 2];
                                    REAL sg = ((tau + nu + ph) & 1) ? (REAL)-1 : (REAL)1;
                                    s += sg * kcoef[j] * R0[((t + tau) * D + (u + nu)) * D + (v + ph)];
                                }
                                S[((t * DS + u) * DS + v) * nkc + k] = s;
                            }
                }
                for (int i = 0; i < na; ++i) {
                    int ax, ay, az;
                    SUF(cart_xyz)(la, i, &ax, &ay, &az);
                    for (int j = 0; j < nb; ++j) {
                        int bxx, byy, bzz;
                        SUF(cart_xyz)(lb, j, &bxx, &byy, &bzz);
                        /* per-axis bra coefficients, differentiated where requested */
                        int aa[3] = {ax, ay, az}, bb[3] = {bxx, byy, bzz};
                        REAL* EE[3] = {Ex, Ey, Ez};
                        REAL* out3[3] = {bx, by, bz};
                        for (int d = 0; d < 3; ++d) {
                            for (int t = 0; t < TE; ++t) {
                                REAL v = EI(EE[d], aa[d], bb[d], t);
                                if (d == dA) {
                                    v = (REAL)2 * a * EI(EE[d], aa[d] + 1, bb[d], t);
                                    if (aa[d] > 0) v -= (REAL)aa[d] * EI(EE[d], aa[d] - 1, bb[d], t);
                                }
                                if (d == dB) {
                                    v = (REAL)2 * b * EI(EE[d], aa[d], bb[d] + 1, t);
                                    if (bb[d] > 0) v -= (REAL)bb[d] * EI(EE[d], aa[d], bb[d] - 1, t);
                                }
                                out3[d][t] = v;
                            }
                        }
                        int tx = aa[0] + bb[0] + (dA == 0) + (dB == 0);
                        int ty = aa[1] + bb[1] + (dA == 1) + (dB == 1);
                        int tz = aa[2] + bb[2] + (dA == 2) + (dB == 2);
                        for (int k = 0; k < nkc; ++k) {
                            REAL s = 0;
                            for (int t = 0; t <= tx; ++t)
                                for (int u = 0; u <= ty; ++u)
                                    for (int v = 0; v <= tz; ++v)
                                        s += bx[t] * by[u] * bz[v] * S[((t * DS + u) * DS + v) * nkc + k];
                            acc[(i * nb + j) * nkc + k] += coef * s;
                        }
                    }
                }
            }
        }
#undef EI
    /* bra projection in working precision */
    int nA = bra_pure ? 2 * la + 1 : na, nB = bra_pure ? 2 * lb + 1 : nb;
    if (bra_pure) {
        const REAL* Ta = Tsph + Toff[la];
        const REAL* Tb = Tsph + Toff[lb];
        for (int A_ = 0; A_ < nA; ++A_)
            for (int B_ = 0; B_ < nB; ++B_)
                for (int k = 0; k < nkc; ++k) {
                    REAL s = 0;
                    for (int i = 0; i < na; ++i) {
                        REAL ta = Ta[A_ * na + i];
                        if (ta == 0) continue;
                        for (int j = 0; j < nb; ++j) {
                            REAL tb = Tb[B_ * nb + j];
                            if (tb == 0) continue;
                            s += ta * tb * acc[(i * nb + j) * nkc + k];
                        }
                    }
                    out[(A_ * nB + B_) * nkc + k] = (double)s;
                }
    } else {
        for (int k = 0; k < na * nb * nkc; ++k) out[k] = (double)acc[k];
    }
    free(acc); free(Ex); free(Ey); free(Ez); free(Rn); free(R0); free(S); free(ktnp); free(kcoef);
    free(bx); free(by); free(bz);
    return 0;
}
