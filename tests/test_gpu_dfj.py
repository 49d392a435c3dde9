"""GPU parity for the DF-J build (Sec. 3): gamma_P = sum (mu nu|P) D_mu nu and
J_mu nu = sum_P (mu nu|P) c_P, against the oracle on the same screened task
list the GPU plan uses (exported with lx3c_dfj_group).

gamma and J are sums of many integrals weighted by D and c, so they are
compared normwise: max|gpu - oracle| <= tol * max|oracle| over each vector /
matrix (the integrals themselves are checked element by element in
test_gpu_eri3c.py).  tol = 1e-12 against the binary128 oracle; 1e-10 against
the FP64 oracle, whose solid-harmonic bra projection loses digits on compact
shells (up to ~1e-9 of a block).
"""
import numpy as np
import pytest

import oracle
from paper_2210_03192_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03192_gb300 as m
    return m


def inputs(cl, seed):
    rng = np.random.default_rng(seed)
    n = int(oracle.ao_offsets(cl.orb)[-1])
    naux = int(oracle.ao_offsets(cl.aux)[-1])
    return W.density(rng, n), rng.standard_normal(naux)


def run_gpu(lx, cl, D, c, tol=1e-12):
    plan = lx.DFJPlan(cl.orb, cl.aux, tol)
    g, J = plan.execute(torch.tensor(D, device="cuda"), torch.tensor(c, device="cuda"))
    torch.cuda.synchronize()
    return plan, g.cpu().numpy(), J.cpu().numpy()


def normwise(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_dfj_small_cluster_binary128(lx):
    cl = W.cluster((2, 2, 1), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=71)
    D, c = inputs(cl, 1)
    plan, g, J = run_gpu(lx, cl, D, c)
    tasks = plan.tasks()
    assert len(tasks) == plan.ntasks
    go, Jo = oracle.dfj(cl.orb, cl.aux, D, c, tasks=tasks, mode="quad")
    assert normwise(g, go) < 1e-12
    assert normwise(J, Jo) < 1e-12
    np.testing.assert_allclose(J, J.T, rtol=0, atol=1e-14 * np.abs(J).max())
    assert np.dot(c, g) == pytest.approx(np.sum(D * J), rel=1e-12)


def test_dfj_16_atoms_full(lx):
    cl = W.cluster((4, 2, 2), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=W.SEED_BASE + 2)
    D, c = inputs(cl, 2)
    plan, g, J = run_gpu(lx, cl, D, c)
    go, Jo = oracle.dfj(cl.orb, cl.aux, D, c, tasks=plan.tasks())
    assert normwise(g, go) < 1e-10
    assert normwise(J, Jo) < 1e-10
    assert np.dot(c, g) == pytest.approx(np.sum(D * J), rel=1e-12)


def test_dfj_screening_keeps_everything_at_zero_tol(lx):
    cl = W.cluster((2, 1, 1), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=72)
    plan = lx.DFJPlan(cl.orb, cl.aux, 0.0)
    nsh = cl.orb.nshell
    assert plan.ntasks == nsh * (nsh + 1) // 2 * cl.aux.nshell


def test_dfj_256_atoms_sampled(lx):
    """256-atom cluster (8x8x4 grid): J blocks of 64 random shell pairs
    and gamma of 3 random ket shells against the FP64 oracle."""
    cl = W.cluster256_dfj()
    D, c = inputs(cl, 3)
    plan, g, J = run_gpu(lx, cl, D, c)
    ao = oracle.ao_offsets(cl.orb)
    aq = oracle.ao_offsets(cl.aux)
    groups = plan.groups()
    rng = np.random.default_rng(9)
    # J rows: random (group, pair)
    sel = []
    for _ in range(64):
        gi = int(rng.integers(len(groups)))
        gr = groups[gi]
        i = int(rng.integers(len(gr["counts"])))
        sel.append((gr, i))
    for gr, i in sel:
        a, b = (int(x) for x in gr["pairs"][i])
        Ps = gr["auxs"][:gr["counts"][i]]
        blocks = oracle.eri3c_triples(cl.orb, cl.aux, [[a, b]] * len(Ps), Ps)
        ref = sum(np.einsum("abP,P->ab", X, c[aq[P]:aq[P + 1]]) for X, P in zip(blocks, Ps))
        # J also receives every other group's (a, b) contributions: collect them
        for gr2 in groups:
            if gr2 is gr:
                continue
            hit = np.where((gr2["pairs"][:, 0] == a) & (gr2["pairs"][:, 1] == b))[0]
            for j in hit:
                Ps2 = gr2["auxs"][:gr2["counts"][j]]
                bl2 = oracle.eri3c_triples(cl.orb, cl.aux, [[a, b]] * len(Ps2), Ps2)
                ref = ref + sum(np.einsum("abP,P->ab", X, c[aq[P]:aq[P + 1]]) for X, P in zip(bl2, Ps2))
        got = J[ao[a]:ao[a + 1], ao[b]:ao[b + 1]]
        assert np.abs(got - ref).max() <= 1e-10 * max(np.abs(ref).max(), 1e-300), (a, b)
    # gamma: three random ket shells of low angular momentum
    for P in rng.choice(np.where(cl.aux.l <= 1)[0], size=3, replace=False):
        trip_pairs, trip_w = [], []
        for gr in groups:
            pos = np.where(gr["auxs"] == P)[0]
            if len(pos) == 0:
                continue
            k = int(pos[0])
            keep = np.where(gr["counts"] > k)[0]
            trip_pairs.append(gr["pairs"][keep])
        pairs = np.concatenate(trip_pairs)
        blocks = oracle.eri3c_triples(cl.orb, cl.aux, pairs, np.full(len(pairs), P))
        ref = np.zeros(2 * cl.aux.l[P] + 1)
        for (a, b), X in zip(pairs, blocks):
            w = 1.0 if a == b else 2.0
            ref += w * np.einsum("abP,ab->P", X, D[ao[a]:ao[a + 1], ao[b]:ao[b + 1]])
        got = g[aq[P]:aq[P + 1]]
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), P
