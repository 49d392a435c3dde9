"""Pins of the oracle's density-fitting metric V_PQ = (P|Q) (no GPU).

The metric (Sec. 1: density fitting; c = V^{-1} gamma) is evaluated by the
oracle as the 3-centre integral (P 1|Q) with 1 = exp(-0 r^2).  Pins: the
(s|s) closed form 2 pi^{5/2} / (a b sqrt(a + b)) F_0(a b / (a + b) R^2) and
the one-step (p|s) form; brute-force quadrature of the defining integral
with the same unit function, projected onto solid harmonics; V = V^T (the
bra goes through the Hermite expansion and the bra projection, the ket
through the Hobson route, so the two triangles come from different code);
positive definiteness of the Coulomb metric; the scaling law
V(s r, zeta / s^2) = s^(lP + lQ + 5) V.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import quadrature as Q
from oracle.solid import solid_matrix
from paper_2210_03192_gb300 import workloads as W

PI = math.pi


def f0(T):
    return 1.0 if T == 0 else 0.5 * math.sqrt(PI / T) * math.erf(math.sqrt(T))


def two_shells(l1, l2, seed, k=(1, 1)):
    rng = np.random.default_rng(seed)
    A, B = rng.uniform(-1.5, 1.5, size=(2, 3))
    e = [np.exp(rng.uniform(np.log(0.2), np.log(6.0), size=n)) for n in k]
    c = [rng.uniform(0.3, 1.0, size=n) for n in k]
    return W.make_basis([l1, l2], list(k), [A, B], np.concatenate(e), np.concatenate(c)), (A, B, e, c)


@pytest.mark.parametrize("seed", range(5))
def test_ss_closed_form(seed):
    aux, (A, B, e, c) = two_shells(0, 0, seed)
    V = oracle.metric(aux)
    a, b = e[0][0], e[1][0]
    ref = c[0][0] * c[1][0] * 2 * PI ** 2.5 / (a * b * math.sqrt(a + b)) * f0(a * b / (a + b) * np.sum((A - B) ** 2))
    assert V[0, 1] == pytest.approx(ref, rel=1e-14)
    aa = c[0][0] ** 2 * 2 * PI ** 2.5 / (a * a * math.sqrt(2 * a))
    assert V[0, 0] == pytest.approx(aa, rel=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_ps_closed_form(seed):
    """(p_i|s) = 2 pi^{5/2}/(a b sqrt(a+b)) (rho/a) (B - A)_i F_1(T), rho = a b/(a+b);
    pure p is ordered (y, z, x)."""
    aux, (A, B, e, c) = two_shells(1, 0, 50 + seed)
    V = oracle.metric(aux)
    a, b = e[0][0], e[1][0]
    rho = a * b / (a + b)
    T = rho * np.sum((A - B) ** 2)
    F1 = (f0(T) - math.exp(-T)) / (2 * T)
    v = c[0][0] * c[1][0] * 2 * PI ** 2.5 / (a * b * math.sqrt(a + b)) * (rho / a) * (B - A) * F1
    np.testing.assert_allclose(V[0:3, 3], [v[1], v[2], v[0]], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("l1,l2", [(1, 1), (2, 3), (4, 2), (3, 3)])
def test_quadrature(l1, l2):
    aux, (A, B, e, c) = two_shells(l1, l2, 100 + 10 * l1 + l2, k=(2, 1))
    ref = Q.eri3c_cart_quadrature(l1, A, e[0], c[0], 0, A, [0.0], [1.0], l2, B, e[1], c[1], n_s=200, n_gh=14)
    pure = np.einsum("Aa,Cc,abc->AC", solid_matrix(l1), solid_matrix(l2), ref)
    V = oracle.metric(aux)
    blk = V[:2 * l1 + 1, 2 * l1 + 1:]
    np.testing.assert_allclose(blk, pure, rtol=0, atol=1e-12 * np.abs(pure).max())


def test_symmetric_positive_definite_and_scaling():
    cl = W.cluster((2, 1, 1), W.ORB_RECIPE_DFJ, [(0, 3, 1), (1, 2, 1), (2, 2, 1), (3, 1, 1), (4, 1, 1), (5, 1, 1),
                                                 (6, 1, 1)], seed=11, exp_lo=0.1, exp_hi=50.0)
    V = oracle.metric(cl.aux)
    assert np.abs(V - V.T).max() <= 1e-13 * np.abs(V).max()
    w = np.linalg.eigvalsh(0.5 * (V + V.T))
    assert w.min() > 0
    # scaling: r -> f r, zeta -> zeta / f^2 multiplies (P|Q) by f^(lP + lQ + 5)
    f = 1.3
    aux = cl.aux
    sc = W.make_basis(aux.l, aux.k, aux.xyz * f, aux.exps / f ** 2, aux.coefs)
    V2 = oracle.metric(sc)
    aq = oracle.ao_offsets(aux)
    lao = np.concatenate([np.full(aq[i + 1] - aq[i], aux.l[i]) for i in range(aux.nshell)])
    ref = V * f ** (lao[:, None] + lao[None, :] + 5)
    assert np.abs(V2 - ref).max() <= 1e-12 * np.abs(ref).max()
