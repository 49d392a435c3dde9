"""Parity at the full per-class sweep sizes, in the launch configuration bench.py
times: every one of the 525 (la, lb <= 4 | lc <= 6, K_ab in {1,3,6}) classes at
4096 pairs x 512 ket shells (Eri3cPlan with the planner's own shapes, as the
bench builds it), with a seeded sample of (pair, ket) blocks per class checked
against the oracle one triple at a time.

Criterion (parity.py): every element within 1e-12 relative or 1e-14 absolute
of the oracle, or within 1e-12 of its block's largest magnitude plus 1e-14;
blocks with an element outside the per-element form are recomputed in
binary128 first.
"""
import numpy as np
import pytest

import oracle
from paper_2210_03192_gb300 import workloads as W

from parity import ATOL, RTOL, within

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NSAMPLE = 96


@pytest.fixture(scope="module")
def lx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03192_gb300 as m
    return m


def check_class(lx, la, lb, lc, K):
    p = W.sweep_class(la, lb, lc, K)
    plan = lx.Eri3cPlan(p.orb, p.aux, p.pairs, p.auxs, bra_pure=True)
    out = plan.execute()
    rng = np.random.default_rng(1000 * (la * 100 + lb * 10 + lc) + K)
    ip = rng.integers(0, p.npair, NSAMPLE)
    iq = rng.integers(0, p.naux, NSAMPLE)
    # always include the first and last pair / ket (tile and list edges)
    ip[:2] = [0, p.npair - 1]
    iq[:2] = [0, p.naux - 1]
    g = out[torch.tensor(ip, device=out.device), torch.tensor(iq, device=out.device)].cpu().numpy()
    torch.cuda.synchronize()
    del out
    o = np.stack(oracle.eri3c_triples(p.orb, p.aux, p.pairs[ip], p.auxs[iq]))
    strict = np.abs(g - o) <= np.maximum(RTOL * np.abs(o), ATOL)
    for b in np.where(~strict.all(axis=(1, 2, 3)))[0]:
        o[b] = oracle.eri3c_triples(p.orb, p.aux, p.pairs[ip[b]:ip[b] + 1], p.auxs[iq[b]:iq[b] + 1], mode="quad")[0]
    strict = np.abs(g - o) <= np.maximum(RTOL * np.abs(o), ATOL)
    ok = within(g, o)
    return ok.all(), 1.0 - strict.mean(), int(ok.size)


def test_sweep_all_classes_full_size_sampled(lx):
    failures = []
    worst = 0.0
    for (la, lb, lc, K) in W.SWEEP_CLASSES:
        ok, miss, n = check_class(lx, la, lb, lc, K)
        worst = max(worst, miss)
        if not ok:
            failures.append(((la, lb, lc, K), miss))
    assert not failures, failures[:10]
