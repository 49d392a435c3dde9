"""GPU parity for the DF-J build (Sec. 3): gamma_P = sum (mu nu|P) D_mu nu and
J_mu nu = sum_P (mu nu|P) c_P, against the oracle on the same screened task
list the GPU plan uses (exported with lx3c_dfj_group).

gamma and J are sums of many integrals weighted by D and c, so they are
compared normwise: max|gpu - oracle| <= tol * max|oracle| over each vector,
matrix or sampled block (the integrals themselves are checked element by
element in test_gpu_eri3c.py).  tol = 1e-12 against the binary128 oracle;
1e-10 against the FP64 oracle, whose solid-harmonic bra projection loses
digits on compact shells (up to ~1e-9 of a block).
"""
import numpy as np
import pytest

import oracle
from paper_2210_03192_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from dfj_sampling import sampled_against_oracle  # noqa: E402


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
    """16-atom cluster of the 256-atom recipe: gamma and J in full against the
    FP64 oracle (normwise 1e-10, the FP64 oracle's own floor), and sampled J
    blocks and gamma entries against the binary128 oracle at 1e-12."""
    cl = W.cluster((4, 2, 2), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=W.SEED_BASE + 2)
    D, c = inputs(cl, 2)
    plan, g, J = run_gpu(lx, cl, D, c)
    go, Jo = oracle.dfj(cl.orb, cl.aux, D, c, tasks=plan.tasks())
    assert normwise(g, go) < 1e-10
    assert normwise(J, Jo) < 1e-10
    assert np.dot(c, g) == pytest.approx(np.sum(D * J), rel=1e-12)
    sampled_against_oracle(cl, plan, D, c, g, J, 24, 4, 16, "quad", 1e-12)


def test_dfj_screening_keeps_everything_at_zero_tol(lx):
    cl = W.cluster((2, 1, 1), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=72)
    plan = lx.DFJPlan(cl.orb, cl.aux, 0.0)
    nsh = cl.orb.nshell
    assert plan.ntasks == nsh * (nsh + 1) // 2 * cl.aux.nshell


def test_dfj_256_atoms_sampled(lx):
    """256-atom cluster (8x8x4 grid): J blocks of 48 random shell pairs and
    gamma of 3 random ket shells against the oracle (binary128 for the J
    blocks, FP64 for the long gamma sums)."""
    cl = W.cluster256_dfj()
    D, c = inputs(cl, 3)
    plan, g, J = run_gpu(lx, cl, D, c)
    sampled_against_oracle(cl, plan, D, c, g, J, 48, 0, 9, "quad", 1e-12)
    sampled_against_oracle(cl, plan, D, c, g, J, 0, 3, 10, "double", 1e-10)


def test_dfj_and_gradient_are_bitwise_reproducible(lx):
    """gamma, J and dE/dR are summed in exact fixed point, so repeated
    executes of one plan agree bit for bit whatever order the tiles finish in."""
    cl = W.cluster((2, 2, 1), W.ORB_RECIPE_SMALL, W.AUX_RECIPE_GRAD, seed=W.SEED_BASE + 50)
    D, c = inputs(cl, 11)
    Dt, ct = torch.tensor(D, device="cuda"), torch.tensor(c, device="cuda")
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12, gradient=True)
    runs = []
    for _ in range(3):
        g, J = plan.execute(Dt, ct)
        G = plan.gradient(Dt, ct)
        torch.cuda.synchronize()
        runs.append((g.cpu().numpy().copy(), J.cpu().numpy().copy(), G.cpu().numpy().copy()))
    for r in runs[1:]:
        for a, b in zip(r, runs[0]):
            assert np.array_equal(a, b)
    assert np.array_equal(runs[0][1], runs[0][1].T)


@pytest.mark.parametrize("shape,recipe_aux", [((2, 2, 1), "dfj"), ((2, 1, 1), "grad")])
def test_dfj_contracted_at_intermediates(lx, shape, recipe_aux):
    """The (e 0|c)-level contraction (LX3C_DFJ_CONTRACT: the pair's bra map
    formed once, D and c contracted before the ket transform, HRR and bra
    transforms) gives the per-integral digestion's gamma and J to rounding,
    and the binary128 oracle's."""
    aux = W.AUX_RECIPE_DFJ if recipe_aux == "dfj" else W.AUX_RECIPE_GRAD
    orb = W.ORB_RECIPE_DFJ if recipe_aux == "dfj" else W.ORB_RECIPE_SMALL
    cl = W.cluster(shape, orb, aux, seed=75)
    D, c = inputs(cl, 12)
    Dt, ct = torch.tensor(D, device="cuda"), torch.tensor(c, device="cuda")
    plain = lx.DFJPlan(cl.orb, cl.aux, 1e-12)
    jeng = lx.DFJPlan(cl.orb, cl.aux, 1e-12, contract=True)
    # launches contract only where that saves flops
    assert jeng.ntasks == plain.ntasks and jeng.flops <= plain.flops
    g0, J0 = plain.execute(Dt, ct)
    g1, J1 = jeng.execute(Dt, ct)
    g0, J0, g1, J1 = (x.cpu().numpy() for x in (g0, J0, g1, J1))
    assert normwise(g1, g0) < 1e-12
    assert normwise(J1, J0) < 1e-12
    np.testing.assert_allclose(J1, J1.T, rtol=0, atol=1e-14 * np.abs(J1).max())
    go, Jo = oracle.dfj(cl.orb, cl.aux, D, c, tasks=jeng.tasks(), mode="quad")
    assert normwise(g1, go) < 1e-12
    assert normwise(J1, Jo) < 1e-12
    # gamma alone, J alone, and the energy path
    g2, _ = jeng.execute(Dt, ct, outputs="gamma")
    _, J2 = jeng.execute(Dt, ct, outputs="J")
    assert np.array_equal(g2.cpu().numpy(), g1) and np.array_equal(J2.cpu().numpy(), J1)
