"""The DF-J screen (the reading of "Schwarz screening at 1e-12"): a triple
(pair, ket) is kept when Q_ab Q_P >= tol, with the library's own factors
(lx3c_schwarz_pair / lx3c_schwarz_aux, host-only calls; Q_ab carries a
safety factor of 20 over an analytic estimate of sqrt(max|(ab|ab)|)).

The oracle evaluates every triple the screen drops, on clusters of the DF-J
recipe (4s3p2d1f orbital, 10s7p5d3f2g1h aux): at tol = 1e-12 every dropped
integral is at most tol, and the screen's effect on gamma and J -- the
dropped triples' contributions, with D = C C^T and c ~ N(0, 1) -- is
reported and bounded."""
import numpy as np
import pytest

import oracle
import paper_2210_03192_gb300 as lx
from paper_2210_03192_gb300 import workloads as W

TOL = 1e-12


def split(cl):
    orb, aux = cl.orb, cl.aux
    pairs = [(a, b) for a in range(orb.nshell) for b in range(a, orb.nshell)]
    qp, qa = lx.schwarz_factors(orb, pairs, aux, range(aux.nshell))
    keep = qp[:, None] * qa[None, :] >= TOL
    return pairs, qp, qa, keep


@pytest.mark.parametrize("shape,spacing,seed", [((4, 1, 1), 3.0, 81), ((2, 2, 1), 1.8, 82), ((3, 1, 1), 4.5, 83)])
def test_dropped_triples_are_below_tolerance(shape, spacing, seed):
    cl = W.cluster(shape, W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=seed, spacing=spacing)
    pairs, qp, qa, keep = split(cl)
    ip, iq = np.nonzero(~keep)
    assert keep.sum() > len(ip) > 500  # the cluster exercises the screen both ways
    blocks = oracle.eri3c_triples(cl.orb, cl.aux, [pairs[i] for i in ip], iq)
    big = np.array([np.abs(x).max() for x in blocks])
    assert big.max() <= TOL, big.max()
    est = qp[ip] * qa[iq]
    assert big[est == 0].max(initial=0.0) == 0.0  # the estimate underflows to 0 only where the integrals do


def test_screening_error_in_gamma_and_J():
    """Contributions of the dropped triples to gamma_P = sum (mu nu|P) D_mu nu
    and J_mu nu = sum_P (mu nu|P) c_P on a 16-atom cluster of the recipe."""
    cl = W.cluster((4, 2, 2), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=W.SEED_BASE + 2)
    pairs, qp, qa, keep = split(cl)
    rng = np.random.default_rng(2)
    n = int(oracle.ao_offsets(cl.orb)[-1])
    D = W.density(rng, n)
    c = rng.standard_normal(int(oracle.ao_offsets(cl.aux)[-1]))
    ip, iq = np.nonzero(~keep)
    tasks = np.stack([[pairs[i][0] for i in ip], [pairs[i][1] for i in ip], iq], axis=1)
    dg, dJ = oracle.dfj(cl.orb, cl.aux, D, c, tasks=tasks)
    # the dropped integrals are below 1e-12; weighted by D (|D| <~ n/5) and
    # summed over the dropped pairs of a ket they stay far below gamma's scale
    assert np.abs(dg).max() <= 1e-9, np.abs(dg).max()
    assert np.abs(dJ).max() <= 1e-10, np.abs(dJ).max()
