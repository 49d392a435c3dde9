"""ORACLE (test infrastructure only): brute-force quadrature of the defining integral.

Used only to pin the McMurchie-Davidson oracle on tiny inputs; it shares no
formula with it beyond the definition of the integral (Appendix A):

    [a b|c] = int int phi_a(r1) phi_b(r1) |r1-r2|^-1 phi_c(r2) dr1 dr2.

Route: write 1/r = (2/sqrt(pi)) int_0^inf exp(-t^2 r^2) dt.  For fixed t the
six-dimensional integral factorises into one two-dimensional Gaussian integral
per Cartesian axis,

    I_x(t) = int int (x1-Ax)^ax (x1-Bx)^bx (x2-Cx)^cx
             exp(-za (x1-Ax)^2 - zb (x1-Bx)^2 - zc (x2-Cx)^2 - t^2 (x1-x2)^2),

which is evaluated exactly by a tensor Gauss-Hermite rule after completing the
square (the integrand is polynomial times Gaussian).  The remaining t integral
is mapped to s in [0,1) by t^2 = rho s^2/(1-s^2) (rho = gamma zc/(gamma+zc)),
where the integrand becomes a polynomial in s^2 times exp(-rho |PC|^2 s^2),
and is done by Gauss-Legendre.
"""
import numpy as np

from .solid import cart_list


def _primitive_cart(la, lb, lc, A, B, C, za, zb, zc, n_s=160, n_gh=12):
    """Primitive Cartesian block [nc(la), nc(lb), nc(lc)] by quadrature."""
    A, B, C = (np.asarray(v, float) for v in (A, B, C))
    g = za + zb
    P = (za * A + zb * B) / g
    mu = za * zb / g
    rho = g * zc / (g + zc)
    d = P - C
    s, ws = np.polynomial.legendre.leggauss(n_s)
    s = 0.5 * (s + 1.0)
    ws = 0.5 * ws
    t2 = rho * s * s / (1.0 - s * s)
    dtds = np.sqrt(rho) * (1.0 - s * s) ** -1.5
    y, wy = np.polynomial.hermite.hermgauss(n_gh)
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    W = np.outer(wy, wy)
    # inverse of M = [[g+t2, -t2], [-t2, zc+t2]] and a factor Cf with Cf Cf^T = M^-1
    det = g * zc + t2 * (g + zc)
    i11 = (zc + t2) / det
    i12 = t2 / det
    i22 = (g + t2) / det
    c11 = np.sqrt(i11)
    c21 = i12 / c11
    c22 = np.sqrt(np.maximum(i22 - c21 * c21, 0.0))
    # per-axis moments table: I[axis][ia][ib][ic][s]
    mom = np.zeros((3, la + 1, lb + 1, lc + 1, n_s))
    for ax in range(3):
        u1c = -(rho / g) * s * s * d[ax]
        u2c = (rho / zc) * s * s * d[ax]
        # u = uc + Cf y ; Cf lower triangular [[c11, 0], [c21, c22]]
        u1 = u1c[:, None, None] + c11[:, None, None] * Y1[None]
        u2 = u2c[:, None, None] + c21[:, None, None] * Y1[None] + c22[:, None, None] * Y2[None]
        x1a = u1 + (P[ax] - A[ax])
        x1b = u1 + (P[ax] - B[ax])
        pref = np.exp(-mu * (A[ax] - B[ax]) ** 2 - rho * s * s * d[ax] ** 2) / np.sqrt(det)
        for i in range(la + 1):
            for j in range(lb + 1):
                for k in range(lc + 1):
                    f = x1a ** i * x1b ** j * u2 ** k
                    mom[ax, i, j, k] = pref * np.einsum("sij,ij->s", f, W)
    out = np.zeros((len(cart_list(la)), len(cart_list(lb)), len(cart_list(lc))))
    for ia, a in enumerate(cart_list(la)):
        for ib, b in enumerate(cart_list(lb)):
            for ic, c in enumerate(cart_list(lc)):
                f = mom[0, a[0], b[0], c[0]] * mom[1, a[1], b[1], c[1]] * mom[2, a[2], b[2], c[2]]
                out[ia, ib, ic] = 2.0 / np.sqrt(np.pi) * np.sum(ws * dtds * f)
    return out


def eri3c_cart_quadrature(la, A, ea, ca, lb, B, eb, cb, lc, C, ec, cc, **kw):
    """Contracted Cartesian (a b|c) block by brute-force quadrature."""
    out = 0.0
    for za, xa in zip(ea, ca):
        for zb, xb in zip(eb, cb):
            for zc, xc in zip(ec, cc):
                out = out + xa * xb * xc * _primitive_cart(la, lb, lc, A, B, C, za, zb, zc, **kw)
    return out


def boys_quadrature(m, T, n=400):
    """F_m(T) = int_0^1 y^{2m} exp(-T y^2) dy by Gauss-Legendre on [0,1]."""
    y, w = np.polynomial.legendre.leggauss(n)
    y = 0.5 * (y + 1.0)
    w = 0.5 * w
    return float(np.sum(w * y ** (2 * m) * np.exp(-T * y * y)))
