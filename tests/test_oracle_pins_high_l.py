"""Pins of the oracle at high angular momentum and for derivative classes (no GPU).

The GPU path runs classes up to (gg|i) (total L = 14) and, for gradients,
derivative classes one quantum higher on the bra.  These pins reach that range
with checks that do not re-use the oracle's own formulas:
  - brute-force quadrature of the defining integral (Appendix A) at total L
    up to 10, compared both as true Cartesian blocks and, after projecting the
    quadrature onto solid harmonics, against the oracle's Hobson-route
    solid-harmonic blocks;
  - exact transformation of all-pure blocks under a rigid rotation, with the
    rotation matrices of the solid harmonics fitted from their values at
    random points (oracle/solid.py only), elementwise, at (4,4|6);
  - permutation, translation and the scaling law s^(la+lb+lc+5) at (4,4|6);
  - derivative blocks: the primitive identity
    d/dA_i phi_a = 2 zeta_a phi_{a+1_i} - a_i phi_{a-1_i} (from the definition
    of a Cartesian Gaussian) evaluated with the oracle's non-derivative
    blocks, a fourth-order finite-difference stencil, and the translational
    sum rule dA + dB + dC = 0 (each centre is differentiated independently).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import quadrature as Q
from oracle.solid import cart_list, solid_matrix
from paper_2210_03192_gb300 import workloads as W


def _basis(ls, exps, coefs, centres):
    return W.make_basis(ls, [len(e) for e in exps], centres, np.concatenate(exps), np.concatenate(coefs))


def _geometry(seed, la, lb, lc, nprim=(2, 1, 1), lo=0.3, hi=3.0, box=1.0):
    rng = np.random.default_rng(seed)
    A, B, C = rng.uniform(-box, box, size=(3, 3))
    ex = [np.exp(rng.uniform(np.log(lo), np.log(hi), size=n)) for n in nprim]
    co = [rng.uniform(0.2, 1.0, size=n) for n in nprim]
    orb = _basis([la, lb], ex[:2], co[:2], [A, B])
    aux = _basis([lc], ex[2:], co[2:], [C])
    return orb, aux, (A, B, C), ex, co


# ------------------------------------------------------------------ brute force at high L
@pytest.mark.parametrize("la,lb,lc", [(3, 3, 3), (4, 2, 3), (2, 2, 6), (4, 3, 3)])
def test_bruteforce_quadrature_high_l(la, lb, lc):
    orb, aux, (A, B, C), ex, co = _geometry(501 + 100 * la + 10 * lb + lc, la, lb, lc)
    ref = Q.eri3c_cart_quadrature(la, A, ex[0], co[0], lb, B, ex[1], co[1], lc, C, ex[2], co[2], n_s=220, n_gh=14)
    l, k, off, xyz, e, c, base = oracle._combined(orb, aux)
    flat, _ = oracle.cart_blocks((l, k, off, xyz, e, c), np.array([[0, 1, 2]], np.int32))
    got = flat.reshape(ref.shape)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * scale)
    # the solid-harmonic (Hobson) ket route and the pure bra against the projected quadrature
    pure = np.einsum("Aa,Bb,Cc,abc->ABC", solid_matrix(la), solid_matrix(lb), solid_matrix(lc), ref)
    X = oracle.eri3c(orb, aux, [[0, 1]], [0], bra_pure=True, mode="quad")[0, 0]
    np.testing.assert_allclose(X, pure, rtol=0, atol=1e-11 * np.abs(pure).max())


# ------------------------------------------------------------------ rotations of pure blocks
def _rotation(seed):
    q = np.random.default_rng(seed).standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def _harmonic_rotation(l, R, seed=0):
    """M with S(R u) = M S(u) for the solid harmonics of degree l, fitted by
    least squares from their values at random points (exact in exact
    arithmetic: S(R u) is a harmonic polynomial of degree l)."""
    u = np.random.default_rng(seed).standard_normal((4 * (2 * l + 1) + 8, 3))
    carts = cart_list(l)
    mono = lambda v: np.stack([v[:, 0] ** a * v[:, 1] ** b * v[:, 2] ** c for a, b, c in carts])
    S = solid_matrix(l) @ mono(u)
    SR = solid_matrix(l) @ mono(u @ R.T)
    M, *_ = np.linalg.lstsq(S.T, SR.T, rcond=None)
    return M.T


@pytest.mark.parametrize("la,lb,lc", [(4, 4, 6), (4, 3, 5), (3, 1, 6)])
def test_rotation_maps_pure_blocks_exactly(la, lb, lc):
    """(R a, R b | R C) = sum M_a M_b M_C (a b|C) element by element."""
    p = W.class_problem(la, lb, lc, 3, 2, 2, 1, 1, box=3.0, exp_lo=0.3, exp_hi=5.0, seed=601 + lc)
    X = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=True, mode="quad")
    R = _rotation(17 + la)
    p.orb.xyz = p.orb.xyz @ R.T
    p.aux.xyz = p.aux.xyz @ R.T
    Y = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=True, mode="quad")
    Ma, Mb, Mc = (_harmonic_rotation(l, R) for l in (la, lb, lc))
    Z = np.einsum("Aa,Bb,Cc,PQabc->PQABC", Ma, Mb, Mc, X)
    s = np.abs(Y).max(axis=(2, 3, 4), keepdims=True)
    assert (np.abs(Y - Z) / s).max() < 1e-12


# ------------------------------------------------------------------ invariances at (4,4|6)
def _problem(la, lb, lc, seed):
    return W.class_problem(la, lb, lc, 3, 2, 2, 2, 1, box=3.0, exp_lo=0.2, exp_hi=20.0, seed=seed)


@pytest.mark.parametrize("la,lb,lc", [(4, 4, 6), (4, 2, 5)])
def test_permutation_translation_scaling_high_l(la, lb, lc):
    p = _problem(la, lb, lc, 700 + la + lc)
    X = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=False, mode="quad")
    s = np.abs(X).max(axis=(2, 3, 4), keepdims=True)
    # (ab|C) = (ba|C) transposed
    Xs = oracle.eri3c(p.orb, p.aux, p.pairs[:, ::-1], p.auxs, bra_pure=False, mode="quad")
    assert (np.abs(X - np.swapaxes(Xs, 2, 3)) / s).max() < 1e-14
    # rigid translation
    shift = np.array([0.7, -1.3, 2.1])
    q = _problem(la, lb, lc, 700 + la + lc)
    q.orb.xyz = q.orb.xyz + shift
    q.aux.xyz = q.aux.xyz + shift
    Y = oracle.eri3c(q.orb, q.aux, q.pairs, q.auxs, bra_pure=False, mode="quad")
    assert (np.abs(X - Y) / s).max() < 1e-13
    # r -> f r, zeta -> zeta / f^2: every integral times f^(la+lb+lc+5)
    f = 1.7
    q = _problem(la, lb, lc, 700 + la + lc)
    q.orb.xyz = q.orb.xyz * f
    q.aux.xyz = q.aux.xyz * f
    q.orb.exps = q.orb.exps / f ** 2
    q.aux.exps = q.aux.exps / f ** 2
    Y = oracle.eri3c(q.orb, q.aux, q.pairs, q.auxs, bra_pure=False, mode="quad")
    assert (np.abs(Y - X * f ** (la + lb + lc + 5)) / (s * f ** (la + lb + lc + 5))).max() < 1e-13


# ------------------------------------------------------------------ derivative classes
def _deriv_blocks(orb, aux, centre, axis, mode="quad"):
    l, k, off, xyz, e, c, base = oracle._combined(orb, aux)
    d = [-1, -1, -1]
    d[centre] = axis
    flat, offs, shapes = oracle.blocks((l, k, off, xyz, e, c), np.array([[0, 1, base[1]]], np.int32), mode,
                                       bra_pure=False, ket_pure=True, dA=d[0], dB=d[1], dC=d[2])
    return flat.reshape(shapes[0])


def _cart_pure_ket(orb, aux, mode="quad"):
    return oracle.eri3c(orb, aux, [[0, 1]], [0], bra_pure=False, mode=mode)[0, 0]


@pytest.mark.parametrize("la,lb,lc", [(3, 2, 4), (4, 4, 5), (1, 3, 6)])
def test_derivative_identity_and_sum_rule(la, lb, lc):
    """d/dA_i (a b|C) = sum_prim [2 za (a+1_i b|C) - a_i (a-1_i b|C)] with
    K=1 shells (so the 2 za factor is the shell's own exponent), and
    dA + dB + dC = 0."""
    orb, aux, (A, B, C), ex, co = _geometry(801 + la + lb + lc, la, lb, lc, nprim=(1, 1, 1), lo=0.3, hi=4.0)
    za = ex[0][0]
    up = _basis([la + 1, lb], ex[:2], co[:2], [A, B])
    hi = _cart_pure_ket(up, aux)
    lo = _cart_pure_ket(_basis([la - 1, lb], ex[:2], co[:2], [A, B]), aux) if la > 0 else None
    ia_up = {a: i for i, a in enumerate(cart_list(la + 1))}
    ia_lo = {a: i for i, a in enumerate(cart_list(la - 1))} if la > 0 else {}
    tot = np.zeros((len(cart_list(la)), len(cart_list(lb)), 2 * lc + 1))
    for axis in range(3):
        dA = _deriv_blocks(orb, aux, 0, axis)
        dB = _deriv_blocks(orb, aux, 1, axis)
        dC = _deriv_blocks(orb, aux, 2, axis)
        ref = np.zeros_like(dA)
        for i, a in enumerate(cart_list(la)):
            ap = list(a)
            ap[axis] += 1
            ref[i] = 2 * za * hi[ia_up[tuple(ap)]]
            if a[axis] > 0:
                am = list(a)
                am[axis] -= 1
                ref[i] -= a[axis] * lo[ia_lo[tuple(am)]]
        s = np.abs(ref).max()
        np.testing.assert_allclose(dA, ref, rtol=0, atol=1e-13 * s)
        np.testing.assert_allclose(dA + dB + dC, 0.0, rtol=0, atol=1e-13 * s)
        tot += np.abs(dA)
    assert tot.max() > 0


@pytest.mark.parametrize("la,lb,lc", [(2, 3, 4), (4, 1, 5)])
def test_derivative_finite_difference(la, lb, lc):
    """Fourth-order central stencil of the oracle's integrals in the position
    of each centre, against its derivative blocks (K=2 contractions)."""
    orb, aux, (A, B, C), ex, co = _geometry(901 + la + lc, la, lb, lc, nprim=(2, 2, 1), lo=0.3, hi=4.0)
    h = 2e-3
    for centre in range(3):
        axis = (centre + 1) % 3
        got = _deriv_blocks(orb, aux, centre, axis)

        def shifted(t):
            cen = [A.copy(), B.copy(), C.copy()]
            cen[centre][axis] += t
            o = _basis([la, lb], ex[:2], co[:2], cen[:2])
            a = _basis([lc], ex[2:], co[2:], cen[2:])
            return _cart_pure_ket(o, a)

        fd = (-shifted(2 * h) + 8 * shifted(h) - 8 * shifted(-h) + shifted(-2 * h)) / (12 * h)
        np.testing.assert_allclose(got, fd, rtol=0, atol=2e-9 * np.abs(got).max())
