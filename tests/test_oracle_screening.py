"""Quality of the DF-J screening estimate (the reading of "identical
screening": keep (pair, ket) when Q_ab Q_P >= tol, with the analytic Q of
lx3c_dfj_plan's header comment restated here).  The oracle evaluates every
triple the estimate drops on a stretched 4-atom cluster of the 256-atom
recipe's shells: the estimate is not a strict bound (it can fall ~11x below
the largest element of a triple, worst for compact same-shell pairs), so at
tol = 1e-12 the dropped integrals must stay below 2e-11."""
import numpy as np

import oracle
from paper_2210_03192_gb300 import workloads as W

TOL = 1e-12


def q_pair(b, sa, sb):
    A, B = b.xyz[sa], b.xyz[sb]
    ab2 = float(((A - B) ** 2).sum())
    q = 0.0
    for i in range(b.k[sa]):
        for j in range(b.k[sb]):
            za, zb = b.exps[b.off[sa] + i], b.exps[b.off[sb] + j]
            g = za + zb
            P = (za * A + zb * B) / g
            q += (abs(b.coefs[b.off[sa] + i] * b.coefs[b.off[sb] + j]) * np.exp(-za * zb / g * ab2)
                  * np.sqrt(2 * np.pi ** 2.5 / (g * g * np.sqrt(2 * g)))
                  * (((P - A) ** 2).sum() + 0.5 / g) ** (0.5 * b.l[sa])
                  * (((P - B) ** 2).sum() + 0.5 / g) ** (0.5 * b.l[sb]))
    return q


def q_aux(b, s):
    z = b.exps[b.off[s]:b.off[s] + b.k[s]]
    c = b.coefs[b.off[s]:b.off[s] + b.k[s]]
    return float(np.sum(np.abs(c) * np.sqrt(2 * np.pi ** 2.5 / (z * z * np.sqrt(2 * z))) * (0.5 / z) ** (0.5 * b.l[s])))


def test_dropped_triples_are_small():
    cl = W.cluster((4, 1, 1), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=81, spacing=3.0)
    orb, aux = cl.orb, cl.aux
    qa = np.array([q_aux(aux, s) for s in range(aux.nshell)])
    pairs, kets, est, kept = [], [], [], 0
    for a in range(orb.nshell):
        for b in range(a, orb.nshell):
            qp = q_pair(orb, a, b)
            for s in range(aux.nshell):
                if qp * qa[s] < TOL:
                    pairs.append((a, b))
                    kets.append(s)
                    est.append(qp * qa[s])
                else:
                    kept += 1
    assert kept > len(kets) > 1000  # the cluster exercises the screen both ways
    blocks = oracle.eri3c_triples(orb, aux, pairs, kets)
    big = np.array([np.abs(x).max() for x in blocks])
    assert big.max() < 20 * TOL, big.max()
    est = np.array(est)
    ok = est > 0
    ratio = big[ok] / est[ok]
    assert ratio.max() < 20, ratio.max()
    assert big[~ok].max(initial=0.0) == 0.0  # estimate underflowed to 0 only where the integrals do
