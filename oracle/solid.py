"""ORACLE (test infrastructure only): real solid harmonics as Cartesian polynomials.

Convention (the paper, Sec. 2.5.1 and Appendix A, names the solid-harmonic ket
but fixes no normalisation or order; this is the reading used throughout):
real regular solid harmonics in Racah normalisation,

    S_{l,m}(r) = sqrt((2 - delta_{m0}) (l-|m|)! / (l+|m|)!)
                 r^l P_l^{|m|}(cos theta) * { cos(|m| phi)  m >= 0
                                             { sin(|m| phi)  m <  0

with P_l^M the associated Legendre function WITHOUT the Condon-Shortley
phase, ordered m = -l..l (l = 1 gives y, z, x).  S_{l,0}(0,0,1) = 1.

Derivation used here (exact rational arithmetic until the final square root):
  P_l^M(t) = (1-t^2)^{M/2} d^M P_l/dt^M,  so
  r^l P_l^M(cos theta) {cos, sin}(M phi)
      = [ r^{l-M} Q(z/r) ] * {Re, Im} (x + i y)^M,   Q = d^M P_l / dt^M,
where r^{l-M} Q(z/r) is a polynomial in z and r^2 = x^2+y^2+z^2 because Q has
the parity of l-M.  P_l comes from its explicit finite sum.  This route is
independent of the closed coefficient formula the GPU library uses.

A solid-harmonic Gaussian S_{l,m}(r-C) exp(-zeta|r-C|^2) is then
sum_c T[m][c] x_C^{c_x} y_C^{c_y} z_C^{c_z} exp(-zeta|r-C|^2) over the
Cartesian components c (x descending, then y descending).
"""
from fractions import Fraction
from functools import lru_cache
from math import comb, factorial, sqrt

import numpy as np


def cart_list(l):
    """Cartesian exponents of shell l in canonical order (x desc, then y desc)."""
    return [(x, y, l - x - y) for x in range(l, -1, -1) for y in range(l - x, -1, -1)]


def _legendre_coeffs(l):
    """P_l(t) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l) t^(l-2k); returns {power: Fraction}."""
    out = {}
    for k in range(l // 2 + 1):
        out[l - 2 * k] = Fraction((-1) ** k * comb(l, k) * comb(2 * l - 2 * k, l), 2 ** l)
    return out


def _derivative(poly, M):
    out = dict(poly)
    for _ in range(M):
        nxt = {}
        for p, c in out.items():
            if p > 0:
                nxt[p - 1] = nxt.get(p - 1, 0) + c * p
        out = nxt
    return {p: c for p, c in out.items() if c != 0}


def _mul(p1, p2):
    out = {}
    for (a, b, c), v in p1.items():
        for (d, e, f), w in p2.items():
            key = (a + d, b + e, c + f)
            out[key] = out.get(key, 0) + v * w
    return {k: v for k, v in out.items() if v != 0}


def _r2_power(s):
    """(x^2+y^2+z^2)^s as {(ex,ey,ez): int}."""
    out = {}
    for i in range(s + 1):
        for j in range(s - i + 1):
            k = s - i - j
            coef = factorial(s) // (factorial(i) * factorial(j) * factorial(k))
            out[(2 * i, 2 * j, 2 * k)] = coef
    return out


@lru_cache(maxsize=None)
def solid_harmonic_poly(l, m):
    """Exact S_{l,m} as ({(ex,ey,ez): Fraction}, norm2) with S = sqrt(norm2) * poly."""
    M = abs(m)
    Q = _derivative(_legendre_coeffs(l), M)
    # r^{l-M} Q(z/r) = sum_j q_j z^j r^{l-M-j}
    zr = {}
    for j, qj in Q.items():
        s2 = l - M - j
        assert s2 % 2 == 0
        for key, c in _r2_power(s2 // 2).items():
            k2 = (key[0], key[1], key[2] + j)
            zr[k2] = zr.get(k2, 0) + qj * c
    # Re / Im of (x + i y)^M
    xy = {}
    for k in range(M + 1):
        if (m >= 0 and k % 2 == 0) or (m < 0 and k % 2 == 1):
            sign = (-1) ** (k // 2)
            xy[(M - k, k, 0)] = Fraction(sign * comb(M, k))
    poly = _mul(zr, xy)
    norm2 = Fraction((2 if M > 0 else 1) * factorial(l - M), factorial(l + M))
    return poly, norm2


@lru_cache(maxsize=None)
def solid_matrix(l):
    """T[m+l][c] (float64): S_{l,m} = sum_c T[m+l][c] x^cx y^cy z^cz."""
    carts = cart_list(l)
    idx = {c: i for i, c in enumerate(carts)}
    T = np.zeros((2 * l + 1, len(carts)))
    for m in range(-l, l + 1):
        poly, norm2 = solid_harmonic_poly(l, m)
        scale = sqrt(norm2.numerator) / sqrt(norm2.denominator)
        for key, c in poly.items():
            T[m + l, idx[key]] = float(c) * scale
    T.setflags(write=False)
    return T


def nsph(l):
    return 2 * l + 1


def ncart(l):
    return (l + 1) * (l + 2) // 2


@lru_cache(maxsize=None)
def solid_matrix_hilo(l):
    """(hi, lo) float64 matrices with hi + lo equal to T[m+l][c] to ~1e-32.

    The exact value is sqrt(norm2) * rational; it is evaluated with 50-digit
    decimal arithmetic and split into two doubles, so that the oracle's
    extended and binary128 modes see the coefficients at their own precision."""
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    carts = cart_list(l)
    idx = {c: i for i, c in enumerate(carts)}
    hi = np.zeros((2 * l + 1, len(carts)))
    lo = np.zeros((2 * l + 1, len(carts)))
    for m in range(-l, l + 1):
        poly, norm2 = solid_harmonic_poly(l, m)
        s = (Decimal(norm2.numerator) / Decimal(norm2.denominator)).sqrt()
        for key, c in poly.items():
            v = s * Decimal(c.numerator) / Decimal(c.denominator)
            h = float(v)
            hi[m + l, idx[key]] = h
            lo[m + l, idx[key]] = float(v - Decimal(h))
    return hi, lo
