"""Several densities in one DF-J build (lx3c_dfj_execute_multi): the
digestion of Sec. 3 for nd <= 8 density matrices and coefficient vectors at
once, as small GEMMs on FP64 tensor-core tiles.  Each density's gamma and J
must equal the single-density build of the same plan (normwise 1e-13: only
the summation order differs) and the binary128 oracle (1e-12)."""
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


def normwise(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("nd", [1, 3, 8])
def test_multi_density_matches_single_and_oracle(lx, nd):
    cl = W.cluster((2, 2, 1), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=73)
    rng = np.random.default_rng(nd)
    n = int(oracle.ao_offsets(cl.orb)[-1])
    naux = int(oracle.ao_offsets(cl.aux)[-1])
    Ds = np.stack([W.density(rng, n) for _ in range(nd)])
    cs = rng.standard_normal((nd, naux))
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12)
    g, J = plan.execute_multi(torch.tensor(Ds, device="cuda"), torch.tensor(cs, device="cuda"))
    torch.cuda.synchronize()
    g, J = g.cpu().numpy(), J.cpu().numpy()
    for k in range(nd):
        g1, J1 = plan.execute(torch.tensor(Ds[k], device="cuda"), torch.tensor(cs[k], device="cuda"))
        assert normwise(g[k], g1.cpu().numpy()) < 1e-13
        assert normwise(J[k], J1.cpu().numpy()) < 1e-13
        np.testing.assert_allclose(J[k], J[k].T, rtol=0, atol=1e-14 * np.abs(J[k]).max())
    k = nd - 1
    go, Jo = oracle.dfj(cl.orb, cl.aux, Ds[k], cs[k], tasks=plan.tasks(), mode="quad")
    assert normwise(g[k], go) < 1e-12
    assert normwise(J[k], Jo) < 1e-12


def test_multi_density_one_output(lx):
    cl = W.cluster((2, 1, 1), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=74)
    rng = np.random.default_rng(9)
    n = int(oracle.ao_offsets(cl.orb)[-1])
    naux = int(oracle.ao_offsets(cl.aux)[-1])
    Ds = torch.tensor(np.stack([W.density(rng, n) for _ in range(4)]), device="cuda")
    cs = torch.tensor(rng.standard_normal((4, naux)), device="cuda")
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12)
    g, J0 = plan.execute_multi(Ds, None, outputs="gamma")
    assert J0 is None
    g2, J = plan.execute_multi(None, cs, outputs="J")
    assert g2 is None
    gb, Jb = plan.execute_multi(Ds, cs)
    assert normwise(g.cpu().numpy(), gb.cpu().numpy()) < 1e-14
    assert normwise(J.cpu().numpy(), Jb.cpu().numpy()) < 1e-14
