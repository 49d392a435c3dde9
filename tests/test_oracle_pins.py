"""Pins of the CPU oracle against things other than itself (no GPU).

Each check below is chosen so that a plausible slip in the oracle (a dropped
term, a wrong sign or index, a transposed operand) fails at least one of them:
closed forms printed in the paper (Sec. 2.5.2), textbook special cases of the
Boys function, brute-force quadrature of the defining integral (Appendix A),
symmetry / invariance / scaling laws of the exact integrals, and a re-run in
extended precision.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import quadrature as Q
from oracle.solid import cart_list, solid_matrix, solid_harmonic_poly
from paper_2210_03192_gb300 import workloads as W

PI = math.pi


def f0_erf(T):
    """F_0(T) = (1/2) sqrt(pi/T) erf(sqrt T) (T > 0), 1 at T = 0."""
    if T == 0:
        return 1.0
    return 0.5 * math.sqrt(PI / T) * math.erf(math.sqrt(T))


# ------------------------------------------------------------------ Boys
@pytest.mark.parametrize("m", range(0, 25))
def test_boys_at_zero(m):
    assert oracle.boys(m, 0.0)[m] == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)


@pytest.mark.parametrize("T", [1e-8, 1e-3, 0.3, 1.0, 4.5, 12.0, 29.0, 29.999, 30.0, 45.0, 117.0, 500.0])
def test_boys_f0_erf(T):
    assert oracle.boys(0, T)[0] == pytest.approx(f0_erf(T), rel=2e-15)


@pytest.mark.parametrize("T", [1e-6, 0.2, 2.0, 9.0, 25.0, 31.0, 60.0, 200.0])
def test_boys_downward_identity(T):
    """(2m+1) F_m = 2T F_{m+1} + exp(-T), checked at every m."""
    F = oracle.boys(20, T)
    for m in range(20):
        lhs = (2 * m + 1) * F[m]
        rhs = 2 * T * F[m + 1] + math.exp(-T)
        assert lhs == pytest.approx(rhs, rel=4e-15)


@pytest.mark.parametrize("T", [0.05, 1.5, 7.0, 20.0, 40.0])
def test_boys_quadrature(T):
    F = oracle.boys(16, T)
    for m in range(17):
        q = Q.boys_quadrature(m, T, n=120)
        assert F[m] == pytest.approx(q, rel=2e-14)


def test_boys_extended_precision_agrees():
    for T in np.linspace(0, 140, 57):
        F = oracle.boys(18, T)
        Fl = oracle.boys(18, T, extended=True)
        np.testing.assert_allclose(F, Fl, rtol=3e-15, atol=0)


# ------------------------------------------------------------------ closed forms
def _one(la, lb, lc, A, B, C, ea, eb, ec, ca=(1.0,), cb=(1.0,), cc=(1.0,)):
    orb = W.make_basis([la, lb], [len(ea), len(eb)], [A, B], np.r_[ea, eb], np.r_[ca, cb])
    aux = W.make_basis([lc], [len(ec)], [C], np.asarray(ec, float), np.asarray(cc, float))
    return orb, aux


def _cart(la, lb, lc, A, B, C, ea, eb, ec, ca=(1.0,), cb=(1.0,), cc=(1.0,), extended=False):
    orb, aux = _one(la, lb, lc, A, B, C, ea, eb, ec, ca, cb, cc)
    l, k, off, xyz, ex, co, base = oracle._combined(orb, aux)
    flat, _ = oracle.cart_blocks((l, k, off, xyz, ex, co), np.array([[0, 1, 2]], np.int32), extended)
    return flat.reshape(len(cart_list(la)), len(cart_list(lb)), len(cart_list(lc)))


def _geom(seed):
    rng = np.random.default_rng(seed)
    A, B, C = rng.uniform(-1.5, 1.5, size=(3, 3))
    za, zb, zc = np.exp(rng.uniform(np.log(0.2), np.log(5.0), size=3))
    return A, B, C, za, zb, zc


def _std(A, B, C, za, zb, zc):
    g = za + zb
    P = (za * A + zb * B) / g
    rho = g * zc / (g + zc)
    K = math.exp(-za * zb / g * np.sum((A - B) ** 2))
    pref = 2 * PI ** 2.5 / (g * zc * math.sqrt(g + zc))
    T = rho * np.sum((P - C) ** 2)
    return g, P, rho, K, pref, T


@pytest.mark.parametrize("seed", range(6))
def test_ssss_closed_form(seed):
    """[00|0] = 2 pi^{5/2}/((g+zc)^{1/2} g zc) exp(-za zb/g AB^2) F_0(rho PC^2)  (Sec. 2.5.2)."""
    A, B, C, za, zb, zc = _geom(seed)
    g, P, rho, K, pref, T = _std(A, B, C, za, zb, zc)
    val = _cart(0, 0, 0, A, B, C, [za], [zb], [zc])[0, 0, 0]
    assert val == pytest.approx(pref * K * f0_erf(T), rel=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_ps_s_and_ss_p_closed_forms(seed):
    """[p_i 0|0] = pref K (PA_i F0 - rho/g PC_i F1);  [00|p_i] = pref K rho/zc PC_i F1
    (one step of VRR1 / VRR2 from [000]^(m), Sec. 2.5.1, with F1 from F0 by the
    upward relation)."""
    A, B, C, za, zb, zc = _geom(100 + seed)
    g, P, rho, K, pref, T = _std(A, B, C, za, zb, zc)
    F0 = f0_erf(T)
    F1 = (F0 - math.exp(-T)) / (2 * T)
    ps = _cart(1, 0, 0, A, B, C, [za], [zb], [zc])[:, 0, 0]
    sp = _cart(0, 0, 1, A, B, C, [za], [zb], [zc])[0, 0, :]
    sps = _cart(0, 1, 0, A, B, C, [za], [zb], [zc])[0, :, 0]
    PA, PB, PC = P - A, P - B, P - C
    np.testing.assert_allclose(ps, pref * K * (PA * F0 - rho / g * PC * F1), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(sps, pref * K * (PB * F0 - rho / g * PC * F1), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(sp, pref * K * (rho / zc) * PC * F1, rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------ brute force
@pytest.mark.parametrize("la,lb,lc", [(0, 0, 0), (1, 0, 0), (0, 1, 1), (1, 1, 1), (2, 0, 1), (2, 1, 2), (1, 2, 3), (2, 2, 2)])
def test_bruteforce_quadrature(la, lb, lc):
    rng = np.random.default_rng(7 + la * 100 + lb * 10 + lc)
    A, B, C = rng.uniform(-1.0, 1.0, size=(3, 3))
    ea = np.exp(rng.uniform(np.log(0.3), np.log(3.0), size=2))
    eb = np.exp(rng.uniform(np.log(0.3), np.log(3.0), size=1))
    ec = np.exp(rng.uniform(np.log(0.3), np.log(3.0), size=2))
    ca, cb, cc = rng.uniform(0.2, 1.0, 2), rng.uniform(0.2, 1.0, 1), rng.uniform(0.2, 1.0, 2)
    ref = Q.eri3c_cart_quadrature(la, A, ea, ca, lb, B, eb, cb, lc, C, ec, cc)
    got = _cart(la, lb, lc, A, B, C, ea, eb, ec, ca, cb, cc)
    scale = np.max(np.abs(ref))
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-13 * scale)


# ------------------------------------------------------------------ invariances
def _problem(la, lb, lc, seed, K=(2, 1, 1), box=3.0):
    return W.class_problem(la, lb, lc, 3, 2, *K, box=box, exp_lo=0.2, exp_hi=20.0, seed=seed)


@pytest.mark.parametrize("la,lb,lc", [(1, 0, 2), (2, 1, 1), (3, 2, 2), (1, 3, 3)])
def test_permutation_symmetry(la, lb, lc):
    """(ab|C) = (ba|C) with the bra indices transposed."""
    p = _problem(la, lb, lc, 11)
    X = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=False)
    Xs = oracle.eri3c(p.orb, p.aux, p.pairs[:, ::-1], p.auxs, bra_pure=False)
    np.testing.assert_allclose(X, np.swapaxes(Xs, 2, 3), rtol=1e-12, atol=1e-13 * np.abs(X).max())


@pytest.mark.parametrize("la,lb,lc", [(2, 1, 2), (3, 3, 1)])
def test_translation_invariance(la, lb, lc):
    p = _problem(la, lb, lc, 12)
    X = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=False)
    shift = np.array([0.7, -1.3, 2.1])
    p.orb.xyz = p.orb.xyz + shift
    p.aux.xyz = p.aux.xyz + shift
    Y = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=False)
    np.testing.assert_allclose(X, Y, rtol=1e-11, atol=1e-13 * np.abs(X).max())


@pytest.mark.parametrize("la,lb,lc", [(1, 1, 2), (2, 3, 1)])
def test_scaling_law(la, lb, lc):
    """r -> s r, zeta -> zeta / s^2 multiplies every integral by s^(la+lb+lc+5)."""
    p = _problem(la, lb, lc, 13)
    X = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=False)
    s = 1.7
    p.orb.xyz = p.orb.xyz * s
    p.aux.xyz = p.aux.xyz * s
    p.orb.exps = p.orb.exps / s ** 2
    p.aux.exps = p.aux.exps / s ** 2
    Y = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=False)
    np.testing.assert_allclose(Y, X * s ** (la + lb + lc + 5), rtol=1e-11, atol=1e-13 * np.abs(Y).max())


def _rotation(seed):
    q = np.random.default_rng(seed).standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


@pytest.mark.parametrize("la,lb,lc", [(1, 1, 1), (2, 1, 3), (3, 2, 2), (2, 2, 4)])
def test_rotation_invariance_pure(la, lb, lc):
    """All-pure blocks transform by orthogonal matrices per shell, so their
    Frobenius norm per (pair, aux) is invariant under a rigid rotation."""
    p = _problem(la, lb, lc, 14)
    X = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=True)
    R = _rotation(5)
    p.orb.xyz = p.orb.xyz @ R.T
    p.aux.xyz = p.aux.xyz @ R.T
    Y = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=True)
    nx = np.sqrt(np.sum(X ** 2, axis=(2, 3, 4)))
    ny = np.sqrt(np.sum(Y ** 2, axis=(2, 3, 4)))
    np.testing.assert_allclose(nx, ny, rtol=1e-11, atol=1e-13 * nx.max())


def test_rotation_about_z_by_quarter_turn_pure_p():
    """A quarter turn about z maps (x, y) -> (-y, x); for pure p ordered (y, z, x)
    the ket block must follow exactly."""
    p = _problem(0, 0, 1, 15, K=(1, 1, 1))
    X = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs)
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    p.orb.xyz = p.orb.xyz @ R.T
    p.aux.xyz = p.aux.xyz @ R.T
    Y = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs)
    # new y = old x, new z = old z, new x = -old y
    np.testing.assert_allclose(Y[..., 0], X[..., 2], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Y[..., 1], X[..., 1], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Y[..., 2], -X[..., 0], rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------ special cases
def test_contraction_linearity():
    """A contracted shell equals the coefficient-weighted sum of its primitives."""
    A, B, C, za, zb, zc = _geom(3)
    ea = np.array([0.4, 1.3, 5.0])
    ca = np.array([0.3, 0.9, 0.5])
    full = _cart(2, 1, 2, A, B, C, ea, [zb], [zc], ca, (0.7,), (0.4,))
    parts = sum(_cart(2, 1, 2, A, B, C, [e], [zb], [zc], (c,), (0.7,), (0.4,)) for e, c in zip(ea, ca))
    np.testing.assert_allclose(full, parts, rtol=1e-14, atol=1e-17)


def test_c_at_p_gives_T_zero():
    """C = P makes T = 0, where every F_m = 1/(2m+1): (ss|s) = pref K."""
    A = np.array([0.1, 0.2, -0.3])
    B = np.array([1.0, -0.5, 0.4])
    za, zb, zc = 1.3, 0.7, 2.2
    P = (za * A + zb * B) / (za + zb)
    g, P, rho, K, pref, T = _std(A, B, P, za, zb, zc)
    assert T == 0.0
    assert _cart(0, 0, 0, A, B, P, [za], [zb], [zc])[0, 0, 0] == pytest.approx(pref * K, rel=1e-15)


@pytest.mark.parametrize("la,lb,lc", [(2, 2, 2), (4, 4, 6), (4, 3, 5)])
def test_extended_precision_bounds_rounding(la, lb, lc):
    p = W.class_problem(la, lb, lc, 2, 2, 2, 2, 1, box=6.0, exp_lo=0.05, exp_hi=1e3, seed=21)
    l, k, off, xyz, ex, co, base = oracle._combined(p.orb, p.aux)
    trip = np.array([[0, 1, base[1]], [2, 3, base[1] + 1]], np.int32)
    d, _ = oracle.cart_blocks((l, k, off, xyz, ex, co), trip)
    e, _ = oracle.cart_blocks((l, k, off, xyz, ex, co), trip, extended=True)
    np.testing.assert_allclose(d, e, rtol=1e-11, atol=1e-14 * np.abs(e).max())


# ------------------------------------------------------------------ solid harmonics
def test_solid_harmonics_low_l_table():
    """Racah-normalised real solid harmonics for l <= 2 (textbook table), order m=-l..l."""
    s3 = math.sqrt(3.0)
    T1 = solid_matrix(1)  # cart order x, y, z
    np.testing.assert_allclose(T1, [[0, 1, 0], [0, 0, 1], [1, 0, 0]], atol=1e-16)
    T2 = solid_matrix(2)  # cart order xx, xy, xz, yy, yz, zz
    ref = np.array([[0, s3, 0, 0, 0, 0],
                    [0, 0, 0, 0, s3, 0],
                    [-0.5, 0, 0, -0.5, 0, 1.0],
                    [0, 0, s3, 0, 0, 0],
                    [s3 / 2, 0, 0, -s3 / 2, 0, 0]])
    np.testing.assert_allclose(T2, ref, atol=1e-15)


@pytest.mark.parametrize("l", range(0, 9))
def test_solid_harmonics_are_harmonic_and_sum_rule(l):
    """Laplacian S_lm = 0 exactly, S_l0(0,0,1) = 1 and sum_m S_lm^2 = r^(2l) exactly."""
    from fractions import Fraction
    total = {}
    for m in range(-l, l + 1):
        poly, norm2 = solid_harmonic_poly(l, m)
        lap = {}
        for (a, b, c), v in poly.items():
            for ax, e in enumerate((a, b, c)):
                if e >= 2:
                    key = [a, b, c]
                    key[ax] -= 2
                    lap[tuple(key)] = lap.get(tuple(key), 0) + v * e * (e - 1)
        assert all(v == 0 for v in lap.values())
        if m == 0:
            assert poly.get((0, 0, l), 0) * norm2 == 1 or (poly.get((0, 0, l), 0) ** 2 * norm2 == 1)
        for (a1, b1, c1), v1 in poly.items():
            for (a2, b2, c2), v2 in poly.items():
                key = (a1 + a2, b1 + b2, c1 + c2)
                total[key] = total.get(key, 0) + norm2 * v1 * v2
    total = {k: v for k, v in total.items() if v != 0}
    from oracle.solid import _r2_power
    assert total == {k: Fraction(v) for k, v in _r2_power(l).items()}


@pytest.mark.parametrize("l", range(0, 7))
def test_solid_harmonics_orthogonal_on_sphere(l):
    """<S_lm, S_lm'> over the unit sphere = 4 pi/(2l+1) delta_mm'."""
    x, w = np.polynomial.legendre.leggauss(2 * l + 4)
    phi = 2 * np.pi * (np.arange(4 * l + 8) + 0.5) / (4 * l + 8)
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct * ct)
    X, Y, Z = st * np.cos(ph), st * np.sin(ph), ct
    wt = (w[:, None] * np.full_like(ph, 2 * np.pi / len(phi))).ravel()
    carts = cart_list(l)
    mono = np.stack([(X ** a * Y ** b * Z ** c).ravel() for a, b, c in carts])
    S = solid_matrix(l) @ mono
    G = (S * wt) @ S.T
    np.testing.assert_allclose(G, 4 * np.pi / (2 * l + 1) * np.eye(2 * l + 1), atol=1e-13)


# ------------------------------------------------------------------ solid-harmonic ket route
def _ss_closed(p, ip, iq, l):
    """(s s|C_lm) = pref K F_l(T) S_lm((rho/zc) PC): the one-term closed form
    (VRR2 of Sec. 2.5.1 with a = 0 has no a_i term), F_l in binary128."""
    a, b = p.pairs[ip]
    c = p.auxs[iq]
    A, B, C = p.orb.xyz[a], p.orb.xyz[b], p.aux.xyz[c]
    za, zb, zc = p.orb.exps[p.orb.off[a]], p.orb.exps[p.orb.off[b]], p.aux.exps[p.aux.off[c]]
    ca, cb, cc = p.orb.coefs[p.orb.off[a]], p.orb.coefs[p.orb.off[b]], p.aux.coefs[p.aux.off[c]]
    g, P, rho, K, pref, T = _std(A, B, C, za, zb, zc)
    X = rho / zc * (P - C)
    Fl = oracle.boys(l, T, mode="quad")[l]
    mono = np.array([X[0] ** e[0] * X[1] ** e[1] * X[2] ** e[2] for e in cart_list(l)])
    return pref * K * ca * cb * cc * Fl * (solid_matrix(l) @ mono)


@pytest.mark.parametrize("lc", [0, 1, 2, 4, 6])
def test_ss_solid_ket_closed_form(lc):
    """Includes compact kets far from the bra (T up to several hundred), where
    projecting true Cartesian kets loses up to eight digits."""
    p = W.class_problem(0, 0, lc, 5, 7, 1, 1, 1, box=6.0, exp_lo=0.1, exp_hi=50.0, seed=1006 + lc)
    X = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs)
    for ip in range(5):
        for iq in range(7):
            ref = _ss_closed(p, ip, iq, lc)
            np.testing.assert_allclose(X[ip, iq, 0, 0], ref, rtol=0, atol=2e-14 * np.abs(ref).max())


@pytest.mark.parametrize("la,lb,lc", [(1, 2, 3), (2, 2, 4), (3, 1, 6)])
def test_ket_routes_agree_in_binary128(la, lb, lc):
    """Hermite (Hobson) ket and projected Cartesian ket are the same integral."""
    p = W.class_problem(la, lb, lc, 3, 4, 2, 1, 1, box=6.0, exp_lo=0.1, exp_hi=50.0, seed=41 + lc)
    X = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=False, mode="quad")
    Y = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=False, mode="quad", ket_route="cartesian")
    s = np.abs(X).max(axis=(2, 3, 4), keepdims=True)
    assert (np.abs(X - Y) / s).max() < 1e-9


@pytest.mark.parametrize("la,lb,lc", [(2, 1, 2), (4, 4, 6), (3, 4, 3)])
def test_precision_modes_agree(la, lb, lc):
    p = W.class_problem(la, lb, lc, 2, 3, 2, 2, 1, box=6.0, exp_lo=0.1, exp_hi=50.0, seed=23 + la)
    q = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, mode="quad")
    e = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, mode="extended")
    d = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, mode="double")
    s = np.abs(q).max(axis=(2, 3, 4), keepdims=True)
    assert (np.abs(e - q) / s).max() < 1e-12
    assert (np.abs(d - q) / s).max() < 1e-8


def test_boys_quad_mode():
    for T in [0.0, 0.7, 12.0, 29.9, 30.0, 85.0, 400.0]:
        np.testing.assert_allclose(oracle.boys(24, T, mode="quad"), oracle.boys(24, T, mode="extended"),
                                   rtol=3e-18, atol=0)
