"""Pins of the oracle's DF-J and gradient drivers (no GPU).

gamma_P = sum_{mu nu} (mu nu|P) D_{mu nu},  J_{mu nu} = sum_P (mu nu|P) c_P
(integral digestion into a DF-J build, Sec. 3).  Checks: both equal a plain
einsum over the full (all ordered AO pairs) integral tensor, c.gamma equals
sum(D * J) (both are c^T I D), and the analytic gradient of E = c^T gamma
matches central finite differences and sums to zero over atoms.
"""
import numpy as np
import pytest

import oracle
from paper_2210_03192_gb300 import workloads as W

ORB = [(0, 2, 2), (1, 1, 2), (2, 1, 1)]
AUX = [(0, 2, 1), (1, 1, 1), (2, 1, 1), (3, 1, 1)]


def small_cluster(seed=5, shape=(2, 1, 1)):
    return W.cluster(shape, ORB, AUX, seed, spacing=1.6, jitter=0.2, exp_lo=0.3, exp_hi=8.0)


def full_tensor(cl):
    """I[mu, nu, P] over all ordered shell pairs (pure everywhere)."""
    ao = oracle.ao_offsets(cl.orb)
    aq = oracle.ao_offsets(cl.aux)
    n, naux = int(ao[-1]), int(aq[-1])
    I = np.zeros((n, n, naux))
    nsh = cl.orb.nshell
    for i in range(nsh):
        for j in range(nsh):
            X = oracle.eri3c_triples(cl.orb, cl.aux, [[i, j]] * cl.aux.nshell, np.arange(cl.aux.nshell))
            for P, blk in enumerate(X):
                I[ao[i]:ao[i + 1], ao[j]:ao[j + 1], aq[P]:aq[P + 1]] = blk
    return I


def test_dfj_matches_full_tensor():
    cl = small_cluster()
    rng = np.random.default_rng(1)
    n = int(oracle.ao_offsets(cl.orb)[-1])
    naux = int(oracle.ao_offsets(cl.aux)[-1])
    D = W.density(rng, n)
    c = rng.standard_normal(naux)
    g, J = oracle.dfj(cl.orb, cl.aux, D, c)
    I = full_tensor(cl)
    np.testing.assert_allclose(g, np.einsum("mnP,mn->P", I, D), rtol=1e-12, atol=1e-12 * np.abs(g).max())
    np.testing.assert_allclose(J, np.einsum("mnP,P->mn", I, c), rtol=1e-12, atol=1e-12 * np.abs(J).max())
    assert np.dot(c, g) == pytest.approx(np.sum(D * J), rel=1e-12)
    np.testing.assert_allclose(J, J.T, rtol=0, atol=1e-13 * np.abs(J).max())


def energy(cl, D, c):
    g, _ = oracle.dfj(cl.orb, cl.aux, D, c)
    return float(np.dot(c, g))


def test_gradient_finite_differences_and_sum_rule():
    cl = small_cluster(seed=9, shape=(3, 1, 1))
    rng = np.random.default_rng(2)
    n = int(oracle.ao_offsets(cl.orb)[-1])
    naux = int(oracle.ao_offsets(cl.aux)[-1])
    D = W.density(rng, n)
    c = rng.standard_normal(naux)
    G = oracle.dfj_grad(cl.orb, cl.aux, D, c, cl.natom)
    assert np.abs(G.sum(axis=0)).max() <= 1e-11 * np.abs(G).max()
    h = 1e-4
    for atom in range(cl.natom):
        for ax in range(3):
            vals = []
            for s in (+1, -1):
                orb = W.make_basis(cl.orb.l, cl.orb.k, cl.orb.xyz.copy(), cl.orb.exps, cl.orb.coefs, cl.orb.atom)
                aux = W.make_basis(cl.aux.l, cl.aux.k, cl.aux.xyz.copy(), cl.aux.exps, cl.aux.coefs, cl.aux.atom)
                orb.xyz[orb.atom == atom, ax] += s * h
                aux.xyz[aux.atom == atom, ax] += s * h
                vals.append(energy(W.Cluster(cl.natom, cl.coords, orb, aux), D, c))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert fd == pytest.approx(G[atom, ax], abs=1e-7 * np.abs(G).max())
